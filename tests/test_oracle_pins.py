"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks the oracle against something the paper or the mathematics fixes:
textbook loops written here independently, closed forms, invariants, the paper's own TTGT
worked example run through a library GEMM, library transposes, and published test vectors
of the two hash functions.  Chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def ints(shape, seed, tid, lo=-4, hi=4):
    return synth.tensor(shape, seed, tid, kind="int", lo=lo, hi=hi)


# ---- textbook special cases, written as plain Python loops -----------------------------------

def test_matmul_triple_loop():
    A, B = ints((3, 5), 1, 0), ints((5, 4), 1, 1)
    C = oracle.einsum("C[i,j] = A[i,k] * B[k,j]", A, B)
    for i in range(3):
        for j in range(4):
            s = 0.0
            for k in range(5):
                s += A[i, k] * B[k, j]
            assert C[i, j] == s


def test_dot_outer_matvec():
    x, y = ints((7,), 2, 0), ints((7,), 2, 1)
    d = oracle.einsum("s[] = x[i] * y[i]", x, y)
    assert d.shape == () and float(d) == sum(x[i] * y[i] for i in range(7))
    o = oracle.einsum("O[i,j] = x[i] * y[j]", x, y)
    assert all(o[i, j] == x[i] * y[j] for i in range(7) for j in range(7))
    M = ints((4, 7), 2, 2)
    v = oracle.einsum("v[r] = M[r,c] * x[c]", M, x)
    assert all(v[r] == sum(M[r, c] * x[c] for c in range(7)) for r in range(4))


def test_brute_force_rank3_by_rank3():
    # C[a,b,c,d] = sum_e A[a,e,b] * B[e,d,c] (the shape of the extent-24 FP64 workload),
    # enumerated over the whole label space at tiny extents.
    ea, eb, ec, ed, ee = 2, 3, 2, 3, 3
    A, B = ints((ea, ee, eb), 3, 0), ints((ee, ed, ec), 3, 1)
    C = oracle.einsum("C[a,b,c,d] = A[a,e,b] * B[e,d,c]", A, B)
    for a, b, c, d in itertools.product(range(ea), range(eb), range(ec), range(ed)):
        assert C[a, b, c, d] == sum(A[a, e, b] * B[e, d, c] for e in range(ee))


def test_column_major_memory_layout():
    # element (i,j) of a column-major 2x3 array sits at linear position i + 2*j
    A = np.asfortranarray(np.arange(6.0).reshape((2, 3), order="F"))
    I = np.asfortranarray(np.eye(3))
    C = oracle.einsum("C[i,j] = A[i,k] * I[k,j]", A, I)
    assert list(np.ravel(C, order="F")) == [0, 1, 2, 3, 4, 5]
    assert C[1, 2] == 5.0


# ---- the paper's TTGT worked example through a library GEMM (Section 2) ----------------------

def test_paper_ttgt_example_against_library_gemm():
    # C[a,b,c,d] = A[a,e,b,f] * B[d,f,c,e]; TA[a,b,e,f] = A_p[i,j], TB[e,f,d,c] = B_p[j,k],
    # C_p[i,k] = TC[a,b,d,c] -> C[a,b,c,d].  Column-major merging: (a,b) -> i with a fastest.
    ea, eb, ec, ed, ee, ef = 3, 4, 2, 5, 3, 2
    A = synth.tensor((ea, ee, eb, ef), 4, 0)
    B = synth.tensor((ed, ef, ec, ee), 4, 1)
    TA = np.transpose(A, (0, 2, 1, 3))            # [a,b,e,f]
    TB = np.transpose(B, (3, 1, 0, 2))            # [e,f,d,c]
    Ap = TA.reshape((ea * eb, ee * ef), order="F")
    Bp = TB.reshape((ee * ef, ed * ec), order="F")
    Cp = Ap @ Bp                                  # library GEMM
    TC = Cp.reshape((ea, eb, ed, ec), order="F")  # [a,b,d,c]
    ref = np.transpose(TC, (0, 1, 3, 2))          # [a,b,c,d]
    C = oracle.einsum("C[a,b,c,d] = A[a,e,b,f] * B[d,f,c,e]", A, B)
    np.testing.assert_allclose(C, ref, rtol=1e-13, atol=1e-13)
    # and exactly on integer data
    Ai, Bi = ints(A.shape, 4, 2), ints(B.shape, 4, 3)
    Api = np.transpose(Ai, (0, 2, 1, 3)).reshape((ea * eb, ee * ef), order="F")
    Bpi = np.transpose(Bi, (3, 1, 0, 2)).reshape((ee * ef, ed * ec), order="F")
    refi = np.transpose((Api @ Bpi).reshape((ea, eb, ed, ec), order="F"), (0, 1, 3, 2))
    assert np.array_equal(oracle.einsum("C[a,b,c,d] = A[a,e,b,f] * B[d,f,c,e]", Ai, Bi), refi)


# ---- closed forms -----------------------------------------------------------------------------

def test_all_ones_gives_product_of_contracted_extents():
    ext = dict(i=3, a=4, j=2, b=3, k=5, c=2)
    A = np.ones((ext["k"], ext["a"], ext["c"], ext["i"]), order="F")
    B = np.ones((ext["c"], ext["b"], ext["k"], ext["j"]), order="F")
    C = oracle.einsum("C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]", A, B)
    assert C.shape == (3, 4, 2, 3) and np.all(C == 10.0)


def test_polynomial_closed_form():
    # A[i,k] = i + k, B[k,j] = j*k  ->  C[i,j] = j * (i*S1 + S2)
    I, K, J = 4, 9, 3
    A = np.asfortranarray(np.add.outer(np.arange(I), np.arange(K)).astype(float))
    B = np.asfortranarray(np.outer(np.arange(K), np.arange(J)).astype(float))
    S1, S2 = K * (K - 1) // 2, (K - 1) * K * (2 * K - 1) // 6
    C = oracle.einsum("C[i,j] = A[i,k] * B[k,j]", A, B)
    expect = np.array([[j * (i * S1 + S2) for j in range(J)] for i in range(I)], dtype=float)
    assert np.array_equal(C, expect)


def test_kronecker_delta_gives_the_transpose_and_pins_perm():
    # C[b,a,c] = A[a,e,b] * delta[e,c]  is A with e renamed c, laid out as (b,a,c):
    # exactly the transpose of A by perm (2,0,1) under out.shape[d] = in.shape[perm[d]].
    A = synth.tensor((4, 5, 3), 5, 0)
    delta = np.asfortranarray(np.eye(5))
    C = oracle.einsum("C[b,a,c] = A[a,e,b] * D[e,c]", A, delta)
    T = oracle.transpose(A, (2, 0, 1))
    assert C.shape == T.shape == (3, 4, 5)
    assert np.array_equal(C, T)


def test_alpha_and_accumulate_forms():
    A, B = ints((3, 4), 6, 0), ints((4, 2), 6, 1)
    base = oracle.einsum("C[i,j] = A[i,k] * B[k,j]", A, B)
    assert np.array_equal(oracle.einsum("C[i,j] = 2.5 * A[i,k] * B[k,j]", A, B), 2.5 * base)
    C0 = ints((3, 2), 6, 2)
    assert np.array_equal(oracle.einsum("C[i,j] += A[i,k] * B[k,j]", A, B, out=C0), C0 + base)
    assert np.array_equal(oracle.einsum("C[i,j] -= A[i,k] * B[k,j]", A, B, out=C0), C0 - base)
    assert np.array_equal(oracle.einsum("C[i,j] = sum_{k} A[i,k] * B[k,j]", A, B), base)
    with pytest.raises(ValueError):
        oracle.einsum("C[i,j] = sum_{j} A[i,k] * B[k,j]", A, B)


# ---- invariants -------------------------------------------------------------------------------

def test_linearity_exact_on_integers():
    A, A2, B = ints((3, 4, 2), 7, 0), ints((3, 4, 2), 7, 1), ints((2, 5, 4), 7, 2)
    e = "C[i,j] = A[i,k,l] * B[l,j,k]"
    lhs = oracle.einsum(e, 3 * A - 2 * A2, B)
    rhs = 3 * oracle.einsum(e, A, B) - 2 * oracle.einsum(e, A2, B)
    assert np.array_equal(lhs, rhs)


def test_relabelling_and_operand_swap():
    # exact on integers; on floats only the summation order differs
    A, B = ints((3, 4, 5), 8, 0), ints((5, 6, 4), 8, 1)
    c1 = oracle.einsum("C[i,j] = A[i,k,l] * B[l,j,k]", A, B)
    c2 = oracle.einsum("Z[x,y] = Q[w,y,v] * P[x,v,w]", B, A)
    assert np.array_equal(c1, c2)
    A, B = synth.tensor((3, 4, 5), 8, 2), synth.tensor((5, 6, 4), 8, 3)
    c1 = oracle.einsum("C[i,j] = A[i,k,l] * B[l,j,k]", A, B)
    c2 = oracle.einsum("Z[x,y] = Q[w,y,v] * P[x,v,w]", B, A)
    np.testing.assert_allclose(c1, c2, rtol=1e-14, atol=1e-14)


def test_multi_operand_equals_pairwise_orders():
    # Section 6: the grouping order changes the operation count, not the result
    A, B, C = ints((3, 2, 2), 9, 0), ints((2, 2, 3, 2), 9, 1), ints((3, 2, 4), 9, 2)
    D = oracle.einsum("D[a,b] = A[a,i,j] * B[i,j,k,l] * C[k,l,b]", A, B, C)
    X = oracle.einsum("X[a,k,l] = A[a,i,j] * B[i,j,k,l]", A, B)
    Y = oracle.einsum("Y[i,j,b] = B[i,j,k,l] * C[k,l,b]", B, C)
    assert np.array_equal(D, oracle.einsum("D[a,b] = X[a,k,l] * C[k,l,b]", X, C))
    assert np.array_equal(D, oracle.einsum("D[a,b] = A[a,i,j] * Y[i,j,b]", A, Y))
    # and against numpy's own contraction on the same data
    assert np.array_equal(D, np.einsum("aij,ijkl,klb->ab", A, B, C))


def test_abs_einsum_is_einsum_of_absolute_values():
    A, B = synth.tensor((3, 4), 10, 0), synth.tensor((4, 5), 10, 1)
    e = "C[i,j] = A[i,k] * B[k,j]"
    ab = oracle.abs_einsum(e, A, B)
    np.testing.assert_allclose(ab, np.abs(A) @ np.abs(B), rtol=1e-14)
    assert np.all(ab >= np.abs(oracle.einsum(e, A, B)) - 1e-15)


def test_sampled_equals_full():
    A, B = synth.tensor((5, 3, 4), 11, 0), synth.tensor((3, 6), 11, 1)
    e = "C[i,j,b] = A[i,k,j] * B[k,b]"
    full = oracle.einsum(e, A, B)
    sel = np.array([0, 7, 29, 44, full.size - 1], dtype=np.int64)
    assert np.array_equal(oracle.einsum_sampled(e, A, B, sel=sel), np.ravel(full, order="F")[sel])


def test_repeated_label_reads_a_diagonal():
    A = ints((4, 4), 12, 0)
    tr = oracle.einsum("t[] = A[i,i]", A, )
    assert float(tr) == float(np.trace(A))


# ---- adjoints ---------------------------------------------------------------------------------

def test_adjoint_dot_product_identity_exact():
    A, B = ints((3, 4, 2), 13, 0), ints((2, 5, 4), 13, 1)
    G = ints((3, 5), 13, 2)
    e = "C[i,j] = A[i,k,l] * B[l,j,k]"
    C = oracle.einsum(e, A, B)
    gA, gB = oracle.grad_exprs(e)
    dA = oracle.einsum(gA, G, B)
    dB = oracle.einsum(gB, G, A)
    inner = float(np.sum(G * C))
    assert inner == float(np.sum(dA * A)) == float(np.sum(dB * B))


def test_gradient_by_central_differences():
    # D is trilinear, so a central difference along one operand is exact up to roundoff.
    A, B, C = synth.tensor((3, 2, 2), 14, 0), synth.tensor((2, 2, 3, 2), 14, 1), \
        synth.tensor((3, 2, 4), 14, 2)
    W = synth.tensor((3, 4), 14, 3)
    e = "D[a,b] = A[a,i,j] * B[i,j,k,l] * C[k,l,b]"
    ops = [A, B, C]

    def loss(xs):
        return float(np.sum(W * oracle.einsum(e, *xs)))

    grads = oracle.grad_exprs(e)
    for x in range(3):
        others = [ops[y] for y in range(3) if y != x]
        g = oracle.einsum(grads[x], W, *others)
        v = synth.tensor(ops[x].shape, 14, 10 + x)
        h = 1e-3
        xp = list(ops); xp[x] = ops[x] + h * v
        xm = list(ops); xm[x] = ops[x] - h * v
        fd = (loss(xp) - loss(xm)) / (2 * h)
        assert abs(fd - float(np.sum(g * v))) <= 1e-11 * max(1.0, abs(fd))


# ---- transposes -------------------------------------------------------------------------------

@pytest.mark.parametrize("perm", list(itertools.permutations(range(4))))
def test_transpose_matches_numpy_and_inverts(perm):
    A = synth.tensor((3, 4, 2, 5), 15, 0)
    T = oracle.transpose(A, perm)
    assert T.tobytes(order="F") == np.asfortranarray(np.transpose(A, perm)).tobytes(order="F")
    inv = np.argsort(perm)
    assert oracle.transpose(T, inv).tobytes(order="F") == A.tobytes(order="F")


def test_transpose_moves_bits():
    raw = synth.raw_bits(16, 0, 0, 2 * 3 * 4)
    A64 = np.asfortranarray(raw.view(np.float64).reshape((2, 3, 4), order="F"))
    A64.reshape(-1, order="A")[:4] = np.array([np.nan, -0.0, 5e-324, np.inf])
    bits_in = np.asfortranarray(np.frombuffer(A64.tobytes(order="F"), dtype=np.uint64)
                                .reshape((2, 3, 4), order="F"))
    T = oracle.transpose(A64, (2, 0, 1))
    bits_out = np.frombuffer(T.tobytes(order="F"), dtype=np.uint64).reshape((4, 2, 3), order="F")
    assert np.array_equal(bits_out, np.transpose(bits_in, (2, 0, 1)))
    A32 = np.asfortranarray(raw.astype(np.uint32).view(np.float32).reshape((4, 6), order="F"))
    T32 = oracle.transpose(A32, (1, 0))
    assert T32.tobytes(order="F") == np.asfortranarray(A32.T).tobytes(order="F")


def test_transpose_sampled_and_rejects_bad_perm():
    A = synth.tensor((3, 4, 5), 17, 0)
    full = np.ravel(oracle.transpose(A, (1, 2, 0)), order="F")
    sel = np.array([0, 5, 59], dtype=np.int64)
    assert np.array_equal(oracle.transpose_sampled(A, (1, 2, 0), sel), full[sel])
    with pytest.raises(ValueError):
        oracle.transpose(A, (0, 0, 1))


# ---- triples reduction and the generators -----------------------------------------------------

def test_fmix32_published_vectors():
    # MurmurHash3_x86_32 of the empty input is fmix32(seed): published vectors for seeds
    # 1 and 0xffffffff are 0x514E28B7 and 0x81F16F39.
    assert oracle.fmix32(0) == 0
    assert oracle.fmix32(1) == 0x514E28B7
    assert oracle.fmix32(0xFFFFFFFF) == 0x81F16F39


def test_splitmix64_published_vector():
    # first outputs of SplitMix64 seeded with 1234567 (state advances by GAMMA before mixing)
    assert synth.mix64_int(1234567 + synth.GAMMA) == 6457827717110365317
    assert synth.mix64_int(1234567 + 2 * synth.GAMMA) == 3203168211198807973


_M32 = 0xFFFFFFFF


def _fmix32(h):
    # the MurmurHash3 finalizer as published, written out here so that the weight pin does not
    # rest on the oracle's own hash
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & _M32
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & _M32
    h ^= h >> 16
    return h


def _factor(key, block, x):
    return (_fmix32((key ^ _fmix32((block * 0x9E3779B9 + x) & _M32)) & _M32) >> 8) * 2.0 ** -23 - 1.0


def test_weight_factor_by_definition():
    assert _fmix32(1) == 0x514E28B7 and _fmix32(0xFFFFFFFF) == 0x81F16F39   # published vectors
    for key, block, x in ((77, 5, 0), (77, 5, 123456), (0xDEADBEEF, 4095, 0xFFFFFFFF), (0, 0, 1)):
        assert oracle.triples_factor(key, block, x) == _factor(key, block, x)
    vals = [oracle.triples_factor(3, 1, x) for x in range(4096)]
    assert min(vals) >= -1.0 and max(vals) < 1.0 and abs(np.mean(vals)) < 0.05


def test_triples_reduce_matches_materialised_block():
    # distinct extents, so that a weight built on the wrong label split or the wrong key fails
    ea, eb, ec, ei, ej, ek, ed = 2, 3, 4, 3, 2, 5, 4
    A = synth.tensor((ed, ea, eb, ei), 18, 0, kind="normal", scale=0.1)
    B = synth.tensor((ec, ed, ej, ek), 18, 1, kind="normal", scale=0.1)
    T = oracle.einsum("T[a,b,c,i,j,k] = A[d,a,b,i] * B[c,d,j,k]", A, B)
    a, b, c, i, j, k = np.indices(T.shape)
    oA = a + ea * b + ea * eb * ec * i                              # labels of A: a, b, i
    oB = ea * eb * c + ea * eb * ec * ei * j + ea * eb * ec * ei * ej * k   # labels of B: c, j, k
    assert np.array_equal(oA + oB, np.arange(T.size).reshape(T.shape, order="F"))
    key, blk = 77, 5
    fa = np.vectorize(lambda x: _factor(key, blk, int(x)))(oA)
    fb = np.vectorize(lambda x: _factor(key ^ _M32, blk, int(x)))(oB)
    s, q = oracle.triples_reduce(A, B, key, blk)
    np.testing.assert_allclose(s, float(np.sum(T * fa * fb)), rtol=1e-13)
    np.testing.assert_allclose(q, float(np.sum(T * T)), rtol=1e-13)
    # the same block under another key or block number gives another s (the weight is keyed)
    assert abs(oracle.triples_reduce(A, B, key + 1, blk)[0] - s) > 1e-6 * np.sqrt(q)
    assert abs(oracle.triples_reduce(A, B, key, blk + 1)[0] - s) > 1e-6 * np.sqrt(q)


def test_golden_fixture_table1_parses():
    # the multi-operand expressions printed in Table 1 parse, and their output labels are the
    # labels that appear exactly once
    path = os.path.join(GOLDEN, "table1_expressions.txt")
    rows = [l.split("|") for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 13
    for rhs, speedup in rows:
        ops = oracle.parse("X[] = " + rhs.strip())[4]
        counts = {}
        for _, ls in ops:
            for l in ls:
                counts[l] = counts.get(l, 0) + 1
        assert all(c in (1, 2) for c in counts.values())
        assert float(speedup) >= 1.0


# ---- fused triples accumulation and energy ----------------------------------------------------

TRI_TERMS = ["T[a,b,c,i,j,k] = X[d,a,b,i] * Y[c,d,j,k]",
             "T[a,b,c,i,j,k] = -0.5 * X[d,c,b,i] * Y[a,d,j,k]",
             "T[a,b,c,i,j,k] = 2.0 * X[d,a,b,k] * Y[c,d,j,i]"]


def _tri_block(ext, seed):
    ops = []
    for t, e in enumerate(TRI_TERMS):
        _, _, _, _, operands = oracle.parse(e)
        ops.append(tuple(synth.tensor(tuple(ext[l] for l in ls), seed, 2 * t + q)
                         for q, (_, ls) in enumerate(operands)))
    eps = [synth.tensor((ext[l],), seed, 10 + q) + (1.5 if l in "abc" else -1.5)
           for q, l in enumerate("abcijk")]
    return ops, eps


def test_triples_energy_brute_force_loops():
    ext = dict(a=2, b=3, c=2, i=2, j=3, k=2, d=2)
    ops, eps = _tri_block(ext, 31)
    signs = [-1, -1, -1, 1, 1, 1]
    E, T = oracle.triples_energy(TRI_TERMS, ops, eps, signs)
    (X1, Y1), (X2, Y2), (X3, Y3) = ops
    e_ref = 0.0
    for a in range(2):
        for b in range(3):
            for c in range(2):
                for i in range(2):
                    for j in range(3):
                        for k in range(2):
                            t = 0.0
                            for d in range(2):
                                t += X1[d, a, b, i] * Y1[c, d, j, k]
                                t += -0.5 * X2[d, c, b, i] * Y2[a, d, j, k]
                                t += 2.0 * X3[d, a, b, k] * Y3[c, d, j, i]
                            assert abs(T[a, b, c, i, j, k] - t) <= 1e-15
                            D = -eps[0][a] - eps[1][b] - eps[2][c] + eps[3][i] + eps[4][j] + eps[5][k]
                            e_ref += t * t / D
    assert abs(E - e_ref) <= 1e-13 * abs(e_ref)
    assert E < 0   # every denominator is negative


def test_triples_energy_cancelling_terms_and_closed_form():
    ext = dict(a=3, b=2, c=4, i=2, j=3, k=2, d=5)
    X = synth.tensor((5, 3, 2, 2), 32, 0)
    Y = synth.tensor((4, 5, 3, 2), 32, 1)
    eps = [np.full(ext[l], 0.25) for l in "abcijk"]
    terms = ["T[a,b,c,i,j,k] = X[d,a,b,i] * Y[c,d,j,k]", "T[a,b,c,i,j,k] = -1.0 * X[d,a,b,i] * Y[c,d,j,k]"]
    E, T = oracle.triples_energy(terms, [(X, Y), (X, Y)], eps, [1, 1, -1, 1, 1, 1])
    assert E == 0.0 and not T.any()
    # d = 1 and outer-product operands: T = x_a x_b x_i y_c y_j y_k; with D = 1 everywhere
    # E = product of the six squared norms
    v = {l: synth.tensor((ext[l],), 33, q) for q, l in enumerate("abcijk")}
    X1 = np.einsum("a,b,i->abi", v["a"], v["b"], v["i"]).reshape((1, 3, 2, 2), order="C")
    Y1 = np.einsum("c,j,k->cjk", v["c"], v["j"], v["k"]).reshape((4, 1, 3, 2), order="C")
    eps1 = [np.full(ext[l], 1.0 / 6.0) for l in "abcijk"]
    E1, _ = oracle.triples_energy(terms[:1], [(np.asfortranarray(X1), np.asfortranarray(Y1))], eps1,
                                  [1] * 6)
    closed = np.prod([float(np.dot(v[l], v[l])) for l in "abcijk"])
    assert abs(E1 - closed) <= 1e-13 * closed
