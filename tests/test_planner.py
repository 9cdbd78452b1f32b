"""Host-side tests of the C ABI: symbol exports, parsing, classification, the TTGT form
enumeration (Section 2 / Section 6) and the multi-operand order (Section 6, Table 1).
No GPU needed: comet_plan does no device work."""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

import paper_2102_06827_gb300 as comet
from paper_2102_06827_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2102_06827_gb300 import build
    build.build()


def test_library_exports_every_declared_symbol():
    header = open(os.path.join(ROOT, "include", "comet.h")).read()
    declared = set(re.findall(r"\b(comet_[a-z_]+)\s*\(", header))
    L = comet.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared <= set(_lib.EXPORTS) | {"comet_plan_opts_default"}
    assert "sm_103a" in comet.version()


def plan(expr, ext, dtype="f64", **kw):
    return comet.Plan(expr, ext, dtype, **kw)


def test_parse_errors_and_codes():
    ext = dict(i=3, j=4, k=5)
    for bad in ["C[i,j] A[i,k]*B[k,j]", "C[i,j = A[i,k]*B[k,j]", "C[i,j] = A[i,k]**B[k,j]",
                "= A[i]", "C[i] = 2.0"]:
        with pytest.raises(comet.CometError) as e:
            plan(bad, ext)
        assert e.value.name == "COMET_ERR_PARSE", bad
    with pytest.raises(comet.CometError) as e:
        plan("C[i,x] = A[i,k]*B[k,j]", ext)
    assert e.value.name == "COMET_ERR_LABEL"
    with pytest.raises(comet.CometError) as e:
        plan("C[i,j] = A[i,k]*B[k,j]", dict(i=3, j=4))
    assert e.value.name == "COMET_ERR_LABEL"
    with pytest.raises(comet.CometError) as e:
        plan("C[i,j] = A[i,k]*B[k,j]", dict(i=3, j=0, k=2))
    assert e.value.name == "COMET_ERR_SHAPE"
    with pytest.raises(comet.CometError) as e:
        plan("C[i,j] = sum_{j} A[i,k]*B[k,j]", ext)
    assert e.value.name == "COMET_ERR_LABEL"


def test_accepted_forms():
    ext = dict(i=3, j=4, k=5, l=2)
    plan("A[i,j] = 2.5 * D[j,i]", ext)                     # ta.copy with alpha
    plan("C[i,k,l] = 0.5 * A[i,j] * B[j,k,l]", ext)         # alpha * contraction
    p = plan("D[i,l] = A[i,j] * B[j,k] * C[k,l]", ext)      # multi-operand
    assert len(p.info["steps"]) == 2
    plan("C(i,j) += A(i,k) * B(k,j)", ext)
    plan("C[i,j] -= sum_{k} A[i,k]*B[k,j]", ext)


def _form_tuples(expr, ext):
    p = plan(expr, ext)
    n = p.info["steps"][0]["n_forms"]
    forms = []
    for k in range(n):
        s = plan(expr, ext, form=k).info["steps"][0]
        forms.append((s["swap"], tuple(s["M"]), tuple(s["N"]), tuple(s["K"])))
    return p.info["steps"][0], forms


def test_ttgt_enumeration_contains_the_papers_form():
    # Section 2: C[a,b,c,d] = A[a,e,b,f]*B[d,f,c,e] -> TA[a,b,e,f], TB[e,f,d,c], C_p = TC[a,b,d,c]
    ext = dict(a=3, b=4, c=5, d=6, e=2, f=7)
    chosen, forms = _form_tuples("C[a,b,c,d] = A[a,e,b,f] * B[d,f,c,e]", ext)
    assert (0, ("a", "b"), ("d", "c"), ("e", "f")) in forms
    # every form uses the same label classes: free(A) = {a,b}, free(B) = {c,d}, K = {e,f}
    for swap, M, N, K in forms:
        assert set(K) == {"e", "f"}
        assert {frozenset(M), frozenset(N)} == {frozenset("ab"), frozenset("cd")}
    assert len(forms) == 2 * 2 * 2 * 2
    # the planner's choice puts the output's stride-1 label first in M
    assert chosen["M"][0] == "a" and chosen["swap"] == 0


def test_ccsd_like_form_choice():
    ext = dict(i=64, j=64, k=64, a=192, b=192, c=192)
    s = plan("C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]", ext, precision="split_bf16").info["steps"][0]
    # the output's stride-1 label leads M, so the epilogue's warp stores are contiguous
    assert s["M"] == ["i", "a"] and set(s["N"]) == {"j", "b"} and s["swap"] == 0
    assert set(s["K"]) == {"k", "c"}
    assert s["eff_store"] == 1.0


def test_flops_and_workspace():
    ext = dict(a=24, b=24, c=24, d=24, e=24)
    p = plan("C[a,b,c,d] = A[a,e,b] * B[e,d,c]", ext)
    assert p.flops == 2 * 24 ** 5
    assert p.workspace_bytes == 0
    ps = plan("C[a,b,c,d] = A[a,e,b] * B[e,d,c]", ext, precision="split_bf16")
    kpad = 24 + (-24) % 8
    assert ps.workspace_bytes >= 3 * 2 * kpad * (576 + 576)


def test_batch_labels():
    # a label on both inputs and the result is a batch label of its step: not merged into M, N
    # or K; the step runs once per batch index
    ext = dict(i=3, j=4, k=5, b=6)
    p = plan("C[i,j,b] = A[i,k,b]*B[k,j,b]", ext)
    st = p.info["steps"][0]
    assert st["batch"] == ["b"] and "b" not in st["M"] + st["N"] + st["K"]
    assert p.flops == 2 * 3 * 4 * 5 * 6
    # a label on three inputs: batch in the first step, contracted in the second
    p = plan("s[] = x[i]*y[i]*z[i]", dict(i=7))
    assert [s["batch"] for s in p.info["steps"]] == [["i"], []]
    assert p.flops == 2 * 7 + 2 * 7
    # batch labels and a multi-operand chain
    p = plan("D[b,i] = A[b,i,j]*B[b,j,k]*C[b,k]", dict(b=4, i=5, j=6, k=7))
    assert all(s["batch"] == ["b"] for s in p.info["steps"])
    with pytest.raises(comet.CometError) as e:
        comet.BatchedPlan("C[i,j,b] = A[i,k,b]*B[k,j,b]", ["i", "j", "k", "b"], [[2, 2, 2, 2]], "f64")
    assert e.value.name == "COMET_ERR_UNSUPPORTED"


def test_private_labels_are_reduced_first():
    # a label on one operand only (and not on the output) is summed inside that operand first
    p = plan("C[i] = A[i,k]", dict(i=3, k=5))
    assert [s["kernel"] for s in p.info["steps"]] == ["reduce"]
    p = plan("C[i,j] = A[i,k,l]*B[k,j]", dict(i=3, j=4, k=5, l=2))
    kinds = [s["kernel"] for s in p.info["steps"]]
    assert kinds[0] == "reduce" and len(kinds) == 2
    assert p.info["steps"][0]["c_labels"] == ["i", "k"]
    p = plan("C[i] = A[i]*B[k]", dict(i=3, k=5))
    assert [s["kernel"] for s in p.info["steps"]] == ["reduce", "gemv"]


def test_emulated_fp64_plans():
    ext = dict(a=24, b=24, c=24, d=24, e=24)
    p = plan("C[a,b,c,d] = A[a,e,b] * B[e,d,c]", ext, "f64", precision="emu_f64")
    assert p.info["precision"] == "emu_f64"
    assert p.info["steps"][0]["kernel"] == "gemm_emu_bf16x6"
    kpad = 24 + (-24) % 8
    assert p.workspace_bytes >= 6 * 2 * kpad * (576 + 576)
    # FP64 storage only; merged contraction length up to 98304; not a batched precision
    with pytest.raises(comet.CometError) as e:
        plan("C[i,j] = A[i,k] * B[k,j]", dict(i=4, j=4, k=4), "f32", precision="emu_f64")
    assert e.value.name == "COMET_ERR_DTYPE"
    plan("C[i,j] = A[i,k] * B[k,j]", dict(i=4, j=4, k=98304), "f64", precision="emu_f64")
    with pytest.raises(comet.CometError) as e:
        plan("C[i,j] = A[i,k] * B[k,j]", dict(i=4, j=4, k=98305), "f64", precision="emu_f64")
    assert e.value.name == "COMET_ERR_UNSUPPORTED"
    with pytest.raises(comet.CometError) as e:
        comet.BatchedPlan("C[a,b] = A[a,k] * B[k,b]", ["a", "b", "k"], [[2, 2, 2]], "f64", precision="emu_f64")
    assert e.value.name == "COMET_ERR_UNSUPPORTED"


# ---- multi-operand order vs an explicit enumeration of every contraction sequence ----------

def _labels_outside(sub, ops, out):
    inside = set().union(*[set(ops[i]) for i in sub])
    outside = set(out).union(*[set(ops[i]) for i in range(len(ops)) if i not in sub])
    return inside & outside


def brute_force_min_flops(ops, out, ext):
    """Minimum total flops over every sequence of pairwise contractions (all binary trees)."""
    best = [float("inf")]

    def rec(items, cost):
        # items: list of (frozenset of operand indices)
        if len(items) == 1:
            best[0] = min(best[0], cost)
            return
        for x, y in itertools.combinations(range(len(items)), 2):
            a, b = items[x], items[y]
            la = _labels_outside(a, ops, out)
            lb = _labels_outside(b, ops, out)
            f = 2.0
            for l in la | lb:
                f *= ext[l]
            rest = [items[z] for z in range(len(items)) if z not in (x, y)]
            rec(rest + [a | b], cost + f)

    rec([frozenset([i]) for i in range(len(ops))], 0.0)
    return best[0]


def _table1_rows():
    rows = []
    for line in open(os.path.join(GOLDEN, "table1_expressions.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        rhs, speedup = line.split("|")
        ops = [t.split(",") for t in re.findall(r"\[([^\]]*)\]", rhs)]
        ops = [[l.strip() for l in o] for o in ops]
        counts = {}
        for o in ops:
            for l in o:
                counts[l] = counts.get(l, 0) + 1
        out = [l for o in ops for l in o if counts[l] == 1]
        rows.append((rhs.strip(), ops, out, float(speedup)))
    return rows


@pytest.mark.parametrize("row", range(13))
def test_table1_order_matches_brute_force(row):
    rhs, ops, out, _ = _table1_rows()[row]
    # occupied labels i,j,m,n small, virtual labels a,b,c,d,e,f large (synthetic extents)
    ext = {l: (16 if l in "ijmn" else 48) for o in ops for l in o}
    expr = f"X[{','.join(out)}] = {rhs}"
    p = plan(expr, ext)
    assert p.flops == pytest.approx(brute_force_min_flops(ops, out, ext), rel=1e-12)
    pn = plan(expr, ext, order="natural")
    assert pn.flops == pytest.approx(p.flops_natural, rel=1e-12)
    assert pn.flops >= p.flops


def test_chain_order_tie_and_workspace_cap():
    # D[a,b] = A[a,i,j] * B[i,j,k,l] * C[k,l,b]: (A.B).C and A.(B.C) both cost 3.02e9 flops
    ext = dict(a=256, b=256, i=48, j=48, k=48, l=48)
    e = "D[a,b] = A[a,i,j] * B[i,j,k,l] * C[k,l,b]"
    p = plan(e, ext, dtype="f32", precision="split_bf16")
    assert p.flops == pytest.approx(2 * 256 * 48 ** 4 + 2 * 256 * 48 ** 2 * 256)
    assert p.info["order"] in ("((A*B)*C)", "(A*(B*C))")
    # an outer product A.C would need 256*48^4*256 elements: excluded by a cap
    pc = plan(e, ext, dtype="f32", workspace_cap=1 << 30)
    assert pc.flops == p.flops
    with pytest.raises(comet.CometError) as err:
        plan(e, ext, dtype="f32", workspace_cap=1024)
    assert err.value.name == "COMET_ERR_WORKSPACE"


def test_transpose_argument_checks():
    import torch
    x = torch.empty(8)
    with pytest.raises(comet.CometError) as e:
        comet.transpose(x, [2, 4], [0, 0], out=torch.empty(8), stream=0)
    assert e.value.name == "COMET_ERR_ARG"


def test_transpose_vector_widths():
    # 16-byte vectors where the leading runs allow, 8-byte ones for FP32 runs of even extent
    # (copy mode: asynchronous 8-byte row pieces), element-wise otherwise (widths in elements;
    # a negative vec_out marks copy mode)
    def step(expr, ext, dtype):
        return comet.Plan(expr, ext, dtype).info["steps"][0]
    t = "C[c,b,d,a] = A[a,b,c,d]"
    s = step(t, dict(a=232, b=16, c=148, d=54), "f32")
    assert (s["kernel"], s["vec_in"], s["vec_out"]) == ("copy", 4, 4)
    s = step(t, dict(a=230, b=16, c=146, d=54), "f32")
    assert (s["vec_in"], s["vec_out"]) == (2, 2) and s["tile"][0] % 2 == 0 and s["tile"][1] % 2 == 0
    s = step(t, dict(a=231, b=16, c=146, d=54), "f32")
    assert (s["vec_in"], s["vec_out"]) == (1, 2)
    s = step(t, dict(a=230, b=16, c=146, d=54), "f64")
    assert (s["vec_in"], s["vec_out"]) == (2, 2)
    # copy mode (the first label stays first): 8-byte pieces for an even FP32 run, element-wise
    # for an odd one
    s = step("C[a,e,d,b,c,f] = A[a,b,c,d,e,f]", dict(a=14, b=30, c=31, d=42, e=62, f=12), "f32")
    assert (s["vec_in"], s["vec_out"]) == (2, -2)
    s = step("C[a,e,d,b,c,f] = A[a,b,c,d,e,f]", dict(a=15, b=30, c=31, d=42, e=62, f=12), "f32")
    assert (s["vec_in"], s["vec_out"]) == (1, -1)
    s = step("C[a,e,d,b,c,f] = A[a,b,c,d,e,f]", dict(a=14, b=30, c=31, d=42, e=62, f=12), "f64")
    assert (s["vec_in"], s["vec_out"]) == (2, -2)   # 16 bytes: FP64's full vector
    s = step("C[a,e,d,b,c,f] = A[a,b,c,d,e,f]", dict(a=16, b=30, c=31, d=42, e=62, f=12), "f32")
    assert (s["vec_in"], s["vec_out"]) == (4, -4)


def test_batched_plan_structure():
    import numpy as np
    import synth
    ext = synth.triples_blocks(64)
    names = ["a", "b", "c", "i", "j", "k", "d"]
    e = "T[a,b,c,i,j,k] = A[d,a,b,i] * B[c,d,j,k]"
    for prec in ("native", "split_bf16"):
        p = comet.BatchedPlan(e, names, ext, "f64", precision=prec)
        info = p.describe()
        assert info["batched"] and info["n_blocks"] == 64
        flops = sum(2.0 * np.prod(r) for r in ext)
        assert p.flops == pytest.approx(flops)
        assert p.num_tiles() == (2 if prec == "split_bf16" else 4)
        if prec == "split_bf16":
            # tcgen05 kernel; K = d <= 32 everywhere, so one accumulator per tile; each operand's
            # planes hold ceil(K/32) chunks x 3 planes x rows rounded up to 256 (rows of 32 values)
            assert info["kernel"] == "tcgen05" and info["dual_accumulators"] == 0
            rows = 0
            for a, b, c, i, j, k, d in ext:
                r = lambda x: -(-x // 256) * 256
                rows += -(-d // 32) * 3 * (r(a * b * i) + r(c * j * k))
            assert info["plane_rows"] == rows
            ext2 = ext.copy()
            ext2[5, 6] = 40   # one block with K = 40: the hh products get their own accumulator
            assert comet.BatchedPlan(e, names, ext2, "f64", precision=prec).describe()["dual_accumulators"] == 1
        for c in range(p.num_tiles()):
            p.set_tile(c)
            assert p.describe()["tile_cfg"] == c
        with pytest.raises(comet.CometError):
            p.set_tile(p.num_tiles())
    with pytest.raises(comet.CometError) as err:
        comet.BatchedPlan("D[a,b] = A[a,i] * B[i,j] * C[j,b]", ["a", "b", "i", "j"], [[2, 2, 2, 2]], "f64")
    assert err.value.name in ("COMET_ERR_UNSUPPORTED", "COMET_ERR_DTYPE")
    with pytest.raises(comet.CometError) as err:
        comet.BatchedPlan(e, names, np.zeros((2, 7), dtype=np.int64), "f64")
    assert err.value.name == "COMET_ERR_SHAPE"


def test_host_pipeline_plans():
    """comet_contract_host slicing: one-step split / emulated plans only, along the last label
    of the larger operand's row group, with every slice starting on a 16-byte boundary."""
    ccsd = "C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]"
    full = dict(i=64, j=64, k=64, a=192, b=192, c=192)
    hp = plan(ccsd, full, "f32", precision="split_bf16").info["host_pipe"]
    assert hp["slices"] > 1 and hp["side"] == "N" and hp["label"] == "j"
    assert hp["model_s"][1] < hp["model_s"][0]
    # slice boundaries cover the label in order; on this layout results go back block by block
    for key, n, ext in (("bounds", hp["slices"], 64), ("w_bounds", hp["w_slices"], 192)):
        b = hp[key]
        assert b[0] == 0 and b[-1] == ext and len(b) == n + 1 and all(x < y for x, y in zip(b, b[1:]))
    assert hp["blockwise"]
    assert "host_pipe" in plan(ccsd, full, "f64", precision="emu_f64").info
    for kw in (dict(precision="native"), dict(precision="split_bf16", host_slices=1)):
        assert "host_pipe" not in plan(ccsd, full, "f32", **kw).info
    chain = "D[i,l] = A[i,j] * B[j,k] * C[k,l]"
    assert "host_pipe" not in plan(chain, dict(i=2048, j=2048, k=2048, l=2048), "f32",
                                   precision="split_bf16").info
    # explicit slice counts: ceil(ext / s) per slice, the last one shorter
    hp = plan(ccsd, dict(i=16, j=18, k=16, a=40, b=48, c=48), "f32", precision="split_bf16",
              host_slices=4).info["host_pipe"]
    assert hp["bounds"] == [0, 5, 10, 15, 18] and hp["slices"] == 4
    # B[k,n] slices of n hold k=5 FP32 values per unit: 3 units = 60 bytes is not 16-aligned
    e = "C[m,n] = A[m,k] * B[k,n]"
    assert "host_pipe" not in plan(e, dict(m=4, n=9, k=5), "f32", precision="split_bf16",
                                   host_slices=3).info
    hp = plan(e, dict(m=4, n=9, k=8), "f32", precision="split_bf16", host_slices=3).info["host_pipe"]
    assert hp["label"] == "n" and hp["bounds"] == [0, 3, 6, 9]


def test_host_n_argument_checks():
    """comet_contract_host_n refuses a call count below 1 and missing pointers before any
    device work (no GPU needed to reach these returns)."""
    import ctypes
    p = plan("C[i,j] = A[i,k] * B[k,j]", dict(i=8, j=8, k=8), "f32", precision="split_bf16")
    L = comet.lib()
    vp = ctypes.c_void_p
    hin = (vp * 2)(16, 32)
    hout = (vp * 1)(48)
    din = (vp * 2)(64, 80)
    assert L.comet_contract_host_n(p._h, 0, hin, hout, din, vp(96), vp(112), None) == 12    # COMET_ERR_ARG
    assert L.comet_contract_host_n(p._h, 1, hin, hout, din, None, vp(112), None) == 7       # COMET_ERR_NULL
    assert L.comet_contract_host_n(p._h, 1, (vp * 2)(16, None), hout, din, vp(96), vp(112), None) == 7
    assert L.comet_contract_host_n(p._h, 1, hin, (vp * 1)(None), din, vp(96), vp(112), None) == 7
    assert L.comet_contract_host_n(None, 1, hin, hout, din, vp(96), vp(112), None) == 7
    # two calls need 2 x n_in host input pointers: the second call's null one is caught
    assert L.comet_contract_host_n(p._h, 2, (vp * 4)(16, 32, 16, None), (vp * 2)(48, 48), din, vp(96), vp(112),
                                   None) == 7


def test_views_and_diagonals_layout():
    """comet_plan_views: strides = stored strides x steps, summed over dimensions that share a
    label (diagonals); offset = sum of lo x stored strides; checks of the view arguments."""
    p = plan("C[i,j] = A[i,k] * B[k,j]", dict(i=4, j=5, k=6), "f32", precision="split_bf16",
             views=[(0, 0, 10, 2, 2), (1, 1, 12, 1, 1), (2, 0, 9, 3, 1)])
    v = {x["tensor"]: x for x in p.info["views"]}
    assert v[0] == {"tensor": 0, "offset": 2, "storage": 60, "strides": {"i": 2, "k": 10}}
    assert v[1] == {"tensor": 1, "offset": 6, "storage": 72, "strides": {"k": 1, "j": 6}}
    assert v[2] == {"tensor": 2, "offset": 3, "storage": 45, "strides": {"i": 1, "j": 9}}
    assert "host_pipe" not in p.info
    # diagonals need no view arguments: A[i,i] has stride 1 + 5 for i
    p = plan("t[] = A[i,i]", dict(i=5))
    assert p.info["views"] == [{"tensor": 0, "offset": 0, "storage": 25, "strides": {"i": 6}}]
    assert p.info["steps"][0]["kernel"] == "reduce"
    p = plan("C[i,j] = A[i,k,k] * B[k,j]", dict(i=4, j=3, k=7))
    assert p.info["views"][0]["strides"] == {"i": 1, "k": 4 + 28}
    p = plan("D[i,i] = A[i,k] * B[k,i]", dict(i=4, k=3))
    assert p.info["steps"][0]["batch"] == ["i"]
    assert p.info["views"] == [{"tensor": 2, "offset": 0, "storage": 16, "strides": {"i": 5}}]
    # a whole dimension given as a view is no view
    p = plan("C[i,j] = A[i,k] * B[k,j]", dict(i=4, j=5, k=6), views=[(0, 0, 4, 0, 1)])
    assert "views" not in p.info
    bad = [([(3, 0, 10, 0, 1)], "COMET_ERR_ARG"), ([(0, 2, 10, 0, 1)], "COMET_ERR_ARG"),
           ([(0, 0, 10, 0, 1), (0, 0, 10, 1, 1)], "COMET_ERR_ARG"),
           ([(0, 0, 10, 0, 4)], "COMET_ERR_SHAPE"), ([(0, 0, 10, 7, 1)], "COMET_ERR_SHAPE"),
           ([(0, 0, 10, -1, 1)], "COMET_ERR_SHAPE"), ([(0, 0, 10, 0, 0)], "COMET_ERR_SHAPE"),
           ([(0, 0, 0, 0, 1)], "COMET_ERR_SHAPE")]
    for views, code in bad:
        with pytest.raises(comet.CometError) as e:
            plan("C[i,j] = A[i,k] * B[k,j]", dict(i=4, j=5, k=6), views=views)
        assert e.value.name == code, views
    with pytest.raises(comet.CometError) as e:
        comet.BatchedPlan("C[i,j] = A[i,k,k] * B[k,j]", ["i", "j", "k"], [[3, 4, 5]], "f64")
    assert e.value.name == "COMET_ERR_UNSUPPORTED"


def test_triples_plans():
    import sys
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from triples_terms import LABELS, SIGNS, terms
    ext = [[5, 6, 7, 3, 4, 5, 9], [8, 8, 8, 8, 8, 8, 40]]
    p = comet.TriplesPlan(terms(), LABELS, ext, SIGNS, "f32")
    info = p.info
    assert info["triples"] and info["terms"] == 9 and info["blocks"] == 2
    # tiles per label of the reported edges (4 for the fixed labels; the owned pair's edges
    # depend on the precision)
    edges = info["tile"]
    assert sorted(edges).count(4) >= 4 and len(edges) == 6
    assert info["tiles"] == sum(int(np.prod([-(-row[q] // edges[q]) for q in range(6)])) for row in ext)
    assert info["flops"] == 9 * 2 * (5 * 6 * 7 * 3 * 4 * 5 * 9 + 8 ** 6 * 40)
    # the owned pair sits on different operands in as many terms as any pair can (6 of 9)
    import oracle

    def split(x, y):
        n = 0
        for t in terms():
            xl = oracle.parse(t)[4][0][1]
            n += (x in xl) != (y in xl)
        return n
    a, b = info["own"]
    best = max(split(x, y) for x, y in itertools.combinations("abcijk", 2))
    assert split("abcijk"[a], "abcijk"[b]) == best == 6
    bad = [
        (["T[a,b,c,i,j,k] = X[d,a,b,i] * Y[c,d,j,k] * Z[d]"], "COMET_ERR_UNSUPPORTED"),   # three operands
        (["T[a,b,c,i,j] = X[d,a,b,i] * Y[c,d,j]"], "COMET_ERR_UNSUPPORTED"),             # five labels
        (["T[a,b,c,i,j,k] = X[d,a,b,i] * Y[c,e,j,k]"], "COMET_ERR_UNSUPPORTED"),         # no shared label
        (["T[a,b,c,i,j,k] = X[a,a,b,i] * Y[c,d,j,k]"], "COMET_ERR_UNSUPPORTED"),         # T label twice
        (["T[a,b,c,i,j,k] = X[d,a,b,i] * Y[c,d,j,k]", "T[b,a,c,i,j,k] = X[d,a,b,i] * Y[c,d,j,k]"],
         "COMET_ERR_LABEL"),                                                            # different T order
        (["T[a,b,c,i,j,k] += X[d,a,b,i] * Y[c,d,j,k]"], "COMET_ERR_UNSUPPORTED"),        # accumulate
        (["T[a,b,c,i,j,k] = X[d,a,b,i] * Y[c,d,j,q]"], "COMET_ERR_LABEL"),               # no column for q
    ]
    for tl, code in bad:
        with pytest.raises(comet.CometError) as e:
            comet.TriplesPlan(tl, LABELS + ["e"], [[4] * 8], SIGNS, "f64")
        assert e.value.name == code, tl
    for ext_bad, code in (([[4, 4, 4, 4, 4, 0, 4]], "COMET_ERR_SHAPE"),):
        with pytest.raises(comet.CometError) as e:
            comet.TriplesPlan(terms(), LABELS, ext_bad, SIGNS, "f64")
        assert e.value.name == code
    with pytest.raises(comet.CometError) as e:
        comet.TriplesPlan(terms(), LABELS, [[4] * 7], [1, 1, 1, 1, 1, 2], "f64")
    assert e.value.name == "COMET_ERR_ARG"
    # a triples plan refuses the contraction entry point (checked before any device work)
    ptrs = (ctypes.c_void_p * 18)(*([16] * 18))
    assert comet.lib().comet_contract(p._h, ptrs, ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 12


def _tc_rows(row):
    # plane rows of one block on the FP32 tensor-core path, counted from the layout's definition:
    # per term and operand, tiles (8 along T label a, 4 along the others) x chunks of 32 summed
    # indices x 3 planes x rows per tile (128 for the operand holding a, 64 for the other)
    import sys
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    from triples_terms import LABELS, terms
    ext = dict(zip(LABELS, row))
    total = 0
    for t in terms():
        for _, labels in oracle.parse(t)[4]:
            tl = [l for l in labels if l != "d"]
            tiles = int(np.prod([-(-ext[l] // (8 if l == "a" else 4)) for l in tl]))
            total += tiles * -(-ext["d"] // 32) * 3 * (128 if "a" in tl else 64)
    return total


def test_triples_tensor_core_layout(monkeypatch):
    # FP32 plans run on the tensor cores: pair-tiles of 8 x 4^5, blocks grouped into batches of at
    # most COMET_TRIPLES_BATCH_ROWS plane rows; a block larger than a batch puts the plan on the
    # FMA kernel; FP64 plans always run on the FMA kernel
    import sys
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from triples_terms import LABELS, SIGNS, terms
    ext = [[5, 6, 7, 3, 4, 5, 9], [8, 8, 8, 8, 8, 8, 40], [9, 10, 11, 13, 2, 3, 33]]
    rows = [_tc_rows(r) for r in ext]
    pair_tiles = sum(-(-r[0] // 8) * int(np.prod([-(-r[q] // 4) for q in range(1, 6)])) for r in ext)
    monkeypatch.delenv("COMET_TRIPLES_BATCH_ROWS", raising=False)
    info = comet.TriplesPlan(terms(), LABELS, ext, SIGNS, "f32").info
    assert info["tensor_core"] and info["batches"] == 1 and info["pair_tiles"] == pair_tiles
    assert info["plane_rows"] == sum(rows)
    assert not comet.TriplesPlan(terms(), LABELS, ext, SIGNS, "f64").info["tensor_core"]
    # a cap that holds the largest block: blocks taken in order into batches while they fit
    cap = max(rows)
    monkeypatch.setenv("COMET_TRIPLES_BATCH_ROWS", str(cap))
    batches, cur, region = 0, None, 0
    for r in rows:
        if cur is None or cur + r > cap:
            batches, cur = batches + 1, 0
        cur += r
        region = max(region, cur)
    assert batches >= 2
    info = comet.TriplesPlan(terms(), LABELS, ext, SIGNS, "f32").info
    assert info["tensor_core"] and info["batches"] == batches and info["plane_rows"] == region
    # a cap below the largest block: the FMA kernel
    monkeypatch.setenv("COMET_TRIPLES_BATCH_ROWS", str(max(rows) - 1))
    assert not comet.TriplesPlan(terms(), LABELS, ext, SIGNS, "f32").info["tensor_core"]
