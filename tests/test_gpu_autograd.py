"""GPU tests of the differentiation form: backward through torch.autograd.Function in which the
adjoint of each contraction is itself a planned contraction (multi-operand adjoints recompute
the intermediates they need).

Workload: D[a,b] = sum_{i,j,k,l} A[a,i,j] * B[i,j,k,l] * C[k,l,b], a,b = 256, i,j,k,l = 48,
FP32 storage, split-BF16 products, operand order chosen by the planner.  Checks:
  - central differences in FP64 (h = 1e-3) along a random direction of each operand, the
    forward evaluations done by the oracle: D is trilinear, so the difference quotient equals
    <G, D(..V..)> up to rounding; relative 1e-5
  - gradients against the FP64 oracle's adjoint contraction, on sampled entries: normwise
    1e-6 (split) and 1e-12 (FP64 path)
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import from_dev, to_dev

pytestmark = pytest.mark.gpu

E = "D[a,b] = A[a,i,j] * B[i,j,k,l] * C[k,l,b]"
EXT = dict(a=256, b=256, i=48, j=48, k=48, l=48)
SHAPES = [(256, 48, 48), (48, 48, 48, 48), (48, 48, 256)]


@pytest.fixture(scope="module")
def ag():
    from paper_2102_06827_gb300 import autograd
    return autograd


@pytest.fixture(scope="module")
def data():
    ops = [synth.tensor(s, 4, t) for t, s in enumerate(SHAPES)]
    G = synth.tensor((256, 256), 4, 9)
    return ops, G


def _grads(ag, ops, G, dtype, precision):
    import torch
    ts = [to_dev(x, dtype).requires_grad_(True) for x in ops]
    D = ag.einsum(E, *ts, precision=precision, layout="col")
    D.backward(to_dev(G, dtype))
    torch.cuda.synchronize()
    return from_dev(D.detach()), [from_dev(t.grad) for t in ts]


def _loss_oracle(ops, G):
    """L = sum G * D(ops) by the FP64 oracle, independent of the library's planner and kernels.
    D is summed in two oracle contractions, X[a,k,l] = A[a,i,j] B[i,j,k,l] and then
    D[a,b] = X[a,k,l] C[k,l,b]: the same sum regrouped (associativity of the Section 2 sum),
    which keeps each evaluation to about 1.5e9 terms."""
    X = oracle.einsum("X[a,k,l] = A[a,i,j] * B[i,j,k,l]", ops[0], ops[1])
    D = oracle.einsum("D[a,b] = X[a,k,l] * C[k,l,b]", X, ops[2])
    return float(np.sum(G * D))


@pytest.mark.parametrize("precision,dtype,tol", [("split_bf16", np.float32, 1e-6), ("native", np.float64, 1e-12)])
def test_gradients_against_oracle(ag, data, precision, dtype, tol):
    ops, G = data
    ops_c = [x.astype(dtype).astype(np.float64) for x in ops]
    D, grads = _grads(ag, ops, G, dtype, precision)
    # forward on sampled outputs
    selD = np.arange(0, 256 * 256, 97, dtype=np.int64)
    refD = oracle.einsum_sampled(E, *ops_c, sel=selD)
    assert np.abs(np.ravel(D, order="F")[selD] - refD).max() / np.abs(refD).max() <= tol
    Gc = G.astype(dtype).astype(np.float64)
    for p, expr in enumerate(oracle.grad_exprs(E)):
        others = [ops_c[t] for t in range(3) if t != p]
        n = grads[p].size
        sel = np.unique(synth.integers(40 + p, 0, 400, 0, n - 1).astype(np.int64))
        ref = oracle.einsum_sampled(expr, Gc, *others, sel=sel)
        got = np.ravel(grads[p], order="F")[sel]
        assert np.abs(got - ref).max() / np.abs(ref).max() <= tol, (precision, p)


def test_gradients_against_central_differences(ag, data):
    ops, G = data
    D, grads = _grads(ag, ops, G, np.float32, "split_bf16")
    ops64 = [x.astype(np.float32).astype(np.float64) for x in ops]
    G64 = G.astype(np.float32).astype(np.float64)
    h = 1e-3
    for p in range(3):
        V = synth.tensor(SHAPES[p], 4, 20 + p)
        plus = list(ops64); plus[p] = ops64[p] + h * V
        minus = list(ops64); minus[p] = ops64[p] - h * V
        fd = (_loss_oracle(plus, G64) - _loss_oracle(minus, G64)) / (2 * h)
        an = float(np.sum(grads[p].astype(np.float64) * V))
        assert abs(an - fd) <= 1e-5 * abs(fd), (p, an, fd)


def test_adjoint_plans_recompute_the_intermediate(ag):
    import paper_2102_06827_gb300 as comet
    # the adjoint of A is a three-operand contraction: planned with its own order, so the
    # product of the other two operands is computed again rather than kept from the forward
    adj = ag.adjoint_expr(E, 0)
    p = comet.Plan(adj, dict(EXT), "f32", precision="split_bf16")
    assert len(p.info["steps"]) == 2
    assert p.flops <= p.flops_natural
