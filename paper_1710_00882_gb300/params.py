"""Tersoff parameter sets and the per-triplet table the C ABI takes.

Table rows follow include/tersoff.h: one row per ordered type triplet
(i, j, k) at index (i*nt + j)*nt + k, 14 float64 fields
{m, gamma, lambda3, c, d, h, n, beta, lambda2, B, R, D, lambda1, A}.

Elements are given by Tersoff's published constants (inner/outer cutoff radii
R1 < S); unlike pairs use Tersoff's multicomponent rules: A and B geometric
means (B scaled by chi), lambda1 and lambda2 arithmetic means, R1 and S
geometric means.  Angular constants and beta, n belong to the central atom i;
row (i, j, k) carries the cutoff of the (i, k) pair, which is the one f_C(r_ik)
in zeta_ij needs.
"""
from dataclasses import dataclass
from math import sqrt

import numpy as np


@dataclass(frozen=True)
class Element:
    name: str
    mass: float      # amu
    A: float         # eV
    B: float         # eV
    lam1: float      # 1/A
    lam2: float      # 1/A
    beta: float
    n: float
    c: float
    d: float
    h: float
    R1: float        # A, start of the f_C taper
    S: float         # A, end of the f_C taper


# silicon, Si(C) constants of Tersoff's multicomponent parametrisation
SILICON = Element("Si", 28.0855, A=1830.8, B=471.18, lam1=2.4799, lam2=1.7322, beta=1.1e-6, n=0.78734,
                  c=100390.0, d=16.217, h=-0.59825, R1=2.7, S=3.0)
# carbon, same parametrisation
CARBON = Element("C", 12.011, A=1393.6, B=346.74, lam1=3.4879, lam2=2.2119, beta=1.5724e-7, n=0.72751,
                 c=38049.0, d=4.3484, h=-0.57058, R1=1.8, S=2.1)

CHI = {frozenset(("Si", "C")): 0.9776}


def _pair_consts(a: Element, b: Element):
    chi = 1.0 if a.name == b.name else CHI.get(frozenset((a.name, b.name)), 1.0)
    r1 = sqrt(a.R1 * b.R1)
    s = sqrt(a.S * b.S)
    return dict(A=sqrt(a.A * b.A), B=chi * sqrt(a.B * b.B), lam1=(a.lam1 + b.lam1) / 2,
                lam2=(a.lam2 + b.lam2) / 2, R=(s + r1) / 2, D=(s - r1) / 2)


def build_table(elements, lambda3=0.0, m=1, gamma=1.0):
    """[nt^3, 14] float64 table for a list of Elements (type index = position)."""
    nt = len(elements)
    rows = []
    for ti, ei in enumerate(elements):
        for tj, ej in enumerate(elements):
            pij = _pair_consts(ei, ej)
            for tk, ek in enumerate(elements):
                pik = _pair_consts(ei, ek)
                rows.append([float(m), gamma, lambda3, ei.c, ei.d, ei.h, ei.n, ei.beta,
                             pij["lam2"], pij["B"], pik["R"], pik["D"], pij["lam1"], pij["A"]])
    return np.array(rows, dtype=np.float64).reshape(nt ** 3, 14)


def masses(elements):
    return np.array([e.mass for e in elements], dtype=np.float64)


def for_species(species, **kw):
    """(table, masses) for a tuple of element names, e.g. ("Si",) or ("Si", "C")."""
    lookup = {"Si": SILICON, "C": CARBON}
    els = [lookup[s] for s in species]
    return build_table(els, **kw), masses(els)
