"""Tersoff parameter tables for the oracle -- test infrastructure only.

Written independently of the product's parameter module: the two tables are
built by separate code and compared only through the energies they produce.

Table layout (one row per ordered type triplet (i, j, k), row index
``(i*nt + j)*nt + k``), 14 fields in this order:
    m, gamma, lambda3, c, d, h, n, beta, lambda2, B, R, D, lambda1, A
Two-body terms of the pair (i, j) read row (i, j, j); zeta(i, j, k) (Eq. 3)
reads row (i, j, k), whose R, D are those of the pair (i, k).

Element values are Tersoff's published parameter sets; cutoffs are given as
R = (R1 + S)/2, D = (S - R1)/2 from Tersoff's inner/outer radii R1, S.
"""
import math

import numpy as np

FIELDS = ("m", "gamma", "lambda3", "c", "d", "h", "n", "beta",
          "lambda2", "B", "R", "D", "lambda1", "A")

# Si(C) set (the silicon set of Tersoff's multicomponent paper); the values the
# 512-atom ... 512,000-atom Si workloads name.
SI = dict(A=1830.8, B=471.18, lambda1=2.4799, lambda2=1.7322, beta=1.1e-6,
          n=0.78734, c=100390.0, d=16.217, h=-0.59825, R1=2.7, S=3.0)
# Carbon set of the same paper, used with SI for 3C-SiC.
C = dict(A=1393.6, B=346.74, lambda1=3.4879, lambda2=2.2119, beta=1.5724e-7,
         n=0.72751, c=38049.0, d=4.3484, h=-0.57058, R1=1.8, S=2.1)
CHI_SIC = 0.9776

MASS = {"Si": 28.0855, "C": 12.011}


def _pair(ei, ej, chi):
    """Tersoff's multicomponent combination rules for the pair (i, j)."""
    A = math.sqrt(ei["A"] * ej["A"])
    B = chi * math.sqrt(ei["B"] * ej["B"])
    lam1 = 0.5 * (ei["lambda1"] + ej["lambda1"])
    lam2 = 0.5 * (ei["lambda2"] + ej["lambda2"])
    R1 = math.sqrt(ei["R1"] * ej["R1"])
    S = math.sqrt(ei["S"] * ej["S"])
    return dict(A=A, B=B, lambda1=lam1, lambda2=lam2, R=0.5 * (R1 + S), D=0.5 * (S - R1))


def table(elements, chi=None, lambda3=0.0, m=1.0, gamma=1.0):
    """Per-triplet table for a list of element dicts.

    chi[(a, b)] scales B of the unlike pair (default 1).  Angular parameters
    (beta, n, c, d, h) come from atom i; A, B, lambda1, lambda2 from the pair
    (i, j); R, D of row (i, j, k) from the pair (i, k).
    """
    nt = len(elements)
    chi = chi or {}
    out = np.zeros((nt, nt, nt, len(FIELDS)))
    for i in range(nt):
        for j in range(nt):
            x = chi.get((i, j), chi.get((j, i), 1.0)) if i != j else 1.0
            pij = _pair(elements[i], elements[j], x)
            for k in range(nt):
                pik = _pair(elements[i], elements[k], 1.0)
                ei = elements[i]
                row = dict(m=m, gamma=gamma, lambda3=lambda3, c=ei["c"], d=ei["d"], h=ei["h"],
                           n=ei["n"], beta=ei["beta"], lambda2=pij["lambda2"], B=pij["B"],
                           R=pik["R"], D=pik["D"], lambda1=pij["lambda1"], A=pij["A"])
                out[i, j, k] = [row[f] for f in FIELDS]
    return out.reshape(nt * nt * nt, len(FIELDS))


def si_table(**kw):
    return table([SI], **kw)


def sic_table(**kw):
    """Types: 0 = Si, 1 = C."""
    return table([SI, C], chi={(0, 1): CHI_SIC}, **kw)


def masses(names):
    return np.array([MASS[n] for n in names], dtype=np.float64)
