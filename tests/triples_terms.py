"""The nine permuted terms of the CCSD(T)-style fused accumulation used by the tests and the
bench: T[a,b,c,i,j,k] += sign * X[d, two of a,b,c, o] * Y[v, d, two of i,j,k], one term per
choice of the virtual label v on Y (c, a or b) and the occupied label o on X (i, j or k); each
choice other than (c, i) is one transposition of the base term and flips the sign.  No arithmetic of the method lives here: only label bookkeeping and seeded
inputs."""
import itertools

import numpy as np

import synth

T_LABELS = "abcijk"
LABELS = list("abcijkd")


def terms():
    out = []
    for (vi, v), (oi, o) in itertools.product(enumerate("cab"), enumerate("ijk")):
        xv = [l for l in "abc" if l != v]
        yo = [l for l in "ijk" if l != o]
        sign = (-1.0) ** ((vi > 0) + (oi > 0))   # each non-base choice is one transposition
        out.append(f"T[a,b,c,i,j,k] = {sign} * X{len(out)}[d,{xv[0]},{xv[1]},{o}] * "
                   f"Y{len(out)}[{v},d,{yo[0]},{yo[1]}]")
    return out


SIGNS = [-1, -1, -1, 1, 1, 1]   # D = e_i + e_j + e_k - e_a - e_b - e_c


def operand_labels(expr):
    import oracle
    _, _, _, _, ops = oracle.parse(expr)
    return [ls for _, ls in ops]


def block_inputs(ext, seed, block, kind="uniform", **kw):
    """Host operands and eps vectors of one block: [(X_p, Y_p)], [eps_a, ..., eps_k]."""
    ops = []
    for p, e in enumerate(terms()):
        ops.append(tuple(synth.tensor(tuple(ext[l] for l in ls), seed, 1000 * block + 2 * p + q, kind=kind, **kw)
                         for q, ls in enumerate(operand_labels(e))))
    # virtual energies in [1, 2), occupied in [-2, -1): every denominator is below -6
    eps = [synth.tensor((ext[l],), seed, 1000 * block + 100 + q) * 0.5 + (1.5 if l in "abc" else -1.5)
           for q, l in enumerate(T_LABELS)]
    return ops, eps
