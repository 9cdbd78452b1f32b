#!/usr/bin/env python
"""Benchmark of the contraction hot path on the CCSD-doubles-like workload
C[i,a,j,b] = sum_{k,c} A[k,a,c,i] * B[c,b,k,j] with o = 64 (i,j,k) and v = 192 (a,b,c).

One step = one comet_contract() of the whole path on resident device tensors: split pre-pass
of both operands into bfloat16 planes, tcgen05 split-BF16 GEMM with the output permutation in
its epilogue.  The FP64 form of the same contraction is timed beside it twice -- native (f64
tensor-core MMA) and emulated on the BF16 tensor cores (six slices) -- and every result is
checked against the CPU FP64 oracle on a sample of outputs (the cpu_baseline leg).  Prints one
JSON line (rank 0).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank runs its own copy of the workload (replicas; no collective on the
data path): value = all ranks' flops / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
import zlib

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

EXPR = "C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]"
EXT = dict(i=64, j=64, k=64, a=192, b=192, c=192)
N_ELEM = 64 * 192 * 192 * 64
SCALE = 1.0 / math.sqrt(64 * 192)
METRIC = "contraction GFLOP/s and fraction of roofline (FP64 vs split-precision) at stated error"
WORKLOAD = "ccsd_doubles_like o=64 v=192: C[i,a,j,b] = sum_{k,c} A[k,a,c,i]*B[c,b,k,j]"


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--emu-steps", type=int, default=5)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", default=None, choices=["split", "f64", "emu", "transpose", "triples", "gemv"],
                    help="run one warm-up and one timed launch of a smaller case (for ncu) and exit")
    ap.add_argument("--pc-extents", default="64,128,128,256", help="transpose profile case extents")
    ap.add_argument("--pc-perm", default="3,1,0,2", help="transpose profile case permutation")
    ap.add_argument("--pc-dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--pc-tile", type=int, default=-1, help="batched tile configuration of --profile-case triples")
    ap.add_argument("--pc-o", type=int, default=0, help="--profile-case split/emu/f64: occupied extent (0 = the case default)")
    ap.add_argument("--pc-v", type=int, default=0, help="--profile-case split/emu/f64: virtual extent (0 = the case default)")
    ap.add_argument("--ablation", action="store_true",
                    help="Table 1 natural vs planned order, and every TTGT form vs the chosen one")
    ap.add_argument("--workload", default="ccsd", choices=["ccsd", "triples", "small", "triples_energy"],
                    help="ccsd: the headline line; triples: the batched workload; triples_energy: the "
                         "fused nine-term accumulation with its energy epilogue (separate JSON lines)")
    ap.add_argument("--triples-no-f64", action="store_true", help="triples: skip the FP64 leg")
    ap.add_argument("--te-blocks", type=int, default=4096, help="triples_energy: blocks")
    ap.add_argument("--te-f64-blocks", type=int, default=64, help="triples_energy: blocks of the FP64 leg")
    ap.add_argument("--peak", default=None, choices=["fp64"],
                    help="measure the FP64 pipe (DFMA and f64 tensor-core MMA probes) and exit")
    ap.add_argument("--sweep", default=None, choices=["transpose"],
                    help="time the transpose sweep (rank-4/rank-6, FP32/FP64, 64 MiB - 2 GiB) and exit")
    return ap.parse_args()


def measure_fp64_peak(repeats: int = 3) -> dict:
    """FP64 throughput on this GPU: each probe kernel of the library (DFMA chains, and f64
    tensor-core MMA chains of three shapes) launched after a warm-up, timed with CUDA events on
    its stream, best of `repeats`.  The peak is the fastest probe: it is the denominator of every
    FP64 roofline fraction in the bench lines."""
    import torch
    import paper_2102_06827_gb300 as comet
    s = torch.cuda.current_stream()
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    res = {}
    for kind, name in comet.FP64_PROBES.items():
        iters = 256
        comet.probe_fp64(kind, iters, sink)   # warm-up (and module load)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = 0.0
        for _ in range(repeats + 1):
            e0.record(s)
            fl = comet.probe_fp64(kind, iters, sink)
            e1.record(s)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if ms < 20.0 and iters < (1 << 20):   # grow the launch to ~50 ms before trusting it
                iters = int(iters * 50.0 / max(ms, 1e-3))
                continue
            best = max(best, fl / (ms * 1e-3) / 1e12)
        res[name] = round(best, 4)
    comet.sync_status()
    peak_name = max(res, key=res.get)
    return {"tflops": res[peak_name], "probe": peak_name, "probes_tflops": res,
            "how": "bench.py FP64 probes (comet_probe_fp64): independent chains, one launch of ~50 ms, "
                   "CUDA events, best of 3"}


def run_peak_fp64(a) -> int:
    import torch
    torch.cuda.set_device(0)
    clocks = ClockSampler(0)
    clocks.start()
    res = measure_fp64_peak()
    res["clocks"] = clocks.stop()
    print(json.dumps({"peak": "fp64", **res}), flush=True)
    return 0


def run_transpose_sweep() -> int:
    """Every case of the sweep: GB/s (read + write bytes / time) against the measured HBM copy
    bandwidth and against a same-run device-to-device copy.  Each result is checked bit for bit
    against the oracle on a seeded sample of outputs (the first and last elements included):
    that is the mode's CPU-baseline leg, timed on the host cores.  The inverse permutation
    applied to the result must also give the input back bit for bit."""
    import numpy as np
    import torch
    import oracle
    import paper_2102_06827_gb300 as comet
    import synth
    dev = torch.device("cuda", 0)
    peaks = measured_peaks() or {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    res = []
    cpu_s, cpu_bytes, n_checked = 0.0, 0, 0
    for name, rank, es, perm, ext in synth.transpose_sweep_cases():
        n = math.prod(ext)
        dt = torch.float32 if es == 4 else torch.float64
        x = synth.torch_uniform(zlib.crc32(name.encode()) & 0xFFFF, 0, n, dev, dtype=dt)
        y = torch.empty_like(x)
        z = torch.empty_like(x)
        for _ in range(2):
            comet.transpose(x, ext, perm, out=y)
        reps = max(3, int(2e9 // (2 * es * n)) + 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            comet.transpose(x, ext, perm, out=y)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps * 1e-3
        e0.record()
        for _ in range(reps):
            z.copy_(x)
        e1.record()
        torch.cuda.synchronize()
        tc = e0.elapsed_time(e1) / reps * 1e-3
        inv = [0] * rank
        for d, p in enumerate(perm):
            inv[p] = d
        comet.transpose(y, [ext[p] for p in perm], inv, out=z)
        comet.sync_status()
        ok = bool(torch.equal(z.view(torch.int32 if es == 4 else torch.int64),
                              x.view(torch.int32 if es == 4 else torch.int64)))
        # the oracle leg: seeded sample of outputs (plus the first and the last), bits compared
        sel = np.unique(np.concatenate([[0, n - 1], synth.integers(
            zlib.crc32(name.encode()) & 0xFFFF, 1, 65536, 0, n - 1).astype(np.int64)]))
        got = y[torch.from_numpy(sel).to(dev)].cpu().numpy()
        host = np.asfortranarray(x.cpu().numpy().reshape(tuple(reversed(ext))).T)
        t0 = time.perf_counter()
        ref = oracle.transpose_sampled(host, perm, sel)
        cpu_s += time.perf_counter() - t0
        cpu_bytes += 2 * es * len(sel)
        n_checked += len(sel)
        oracle_ok = got.tobytes() == ref.tobytes()
        gbs = 2 * es * n / t / 1e9
        res.append({"case": name, "perm": perm, "extents": ext, "bytes": es * n, "gbs": round(gbs, 1),
                    "frac": round(gbs / hbm, 4), "memcpy_gbs": round(2 * es * n / tc / 1e9, 1),
                    "bit_exact_oracle": oracle_ok, "oracle_samples": len(sel), "bit_exact_inverse": ok})
        del x, y, z, host
    fr = sorted(r["frac"] for r in res)
    print(json.dumps({"sweep": "transpose", "cases": len(res), "hbm_gbs": hbm,
                      "frac_min": fr[0], "frac_median": fr[len(fr) // 2], "frac_max": fr[-1],
                      "cases_at_or_above_0.70": sum(f >= 0.70 for f in fr),
                      "all_bit_exact_oracle": all(r["bit_exact_oracle"] for r in res),
                      "all_bit_exact_inverse": all(r["bit_exact_inverse"] for r in res),
                      "cpu_baseline": {"value": cpu_bytes / max(cpu_s, 1e-9) / 1e9, "unit": "GB/s",
                                       "cores": oracle.threads(), "kind": "oracle",
                                       "sample": f"{n_checked} sampled outputs over {len(res)} cases "
                                                 "(each case: its first and last outputs and 65536 seeded ones)"},
                      "results": res}))
    return 0


def run_triples(a) -> int:
    """The batched triples workload: 4096 blocks T[a,b,c,i,j,k] = sum_d A[d,a,b,i] * B[c,d,j,k],
    every extent uniform in 8..32 (seed 3), inputs normal(0, 0.1); one launch sequence per step
    (abs-max, split pre-pass, the persistent kernel) inside a captured CUDA graph, reduce epilogue
    (s_b, q_b), tiles chosen by the autotuner.  The CPU baseline leg runs the oracle on the
    smallest, the median and the largest block (timed) and states the error of the GPU's s_b and
    q_b against it.  Prints one JSON line (not the headline line)."""
    import numpy as np
    import torch
    import paper_2102_06827_gb300 as comet
    import synth
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from batched_data import EXPR as TEXPR, LABELS, Blocks, shapes
    ext = synth.triples_blocks(4096)
    peaks = measured_peaks() or {}
    fp64_peak = measure_fp64_peak()
    fl = 2.0 * np.prod(ext, axis=1)
    order = np.argsort(fl, kind="stable")
    check = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    out = {"workload": "batched triples: 4096 blocks, extents uniform 8..32 (seed 3), normal(0,0.1)",
           "flops": float(np.sum(fl))}
    legs = [("split_bf16", np.float32, "f32", a.steps)] + ([] if a.triples_no_f64 else [("native", np.float64, "f64", 1)])
    for prec, dtype, dt, steps in legs:
        blocks = Blocks(ext, dtype, exact_blocks=check)
        plan = comet.BatchedPlan(TEXPR, LABELS, ext, dt, precision=prec)
        ws = plan.workspace()
        plan.prepare(ws)
        res = torch.zeros(2 * blocks.n, dtype=torch.float64, device="cuda")
        ms, best = plan.autotune(blocks.ptrs, res, ws, sample_blocks=0 if prec == "split_bf16" else 96)
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            plan.contract(blocks.ptrs, res, ws, mode=0, key=1, stream=s)
        g.replay()
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        ck = clocks.stop()
        comet.sync_status()
        t = e0.elapsed_time(e1) / steps
        gf = plan.flops / (t * 1e-3) / 1e9
        info = plan.describe()
        entry = {"ms_per_step": t, "gflops": gf, "steps": steps, "tile_times_ms": ms, "tile_cfg": best,
                 "tile": info["tile"], "kernel": info.get("kernel"), "graph": True, "clocks": ck}
        # kernel-only times (eager launches, library profiler)
        comet.profile_enable(True)
        comet.profile_read()
        n_prof = 2 if prec == "split_bf16" else 1
        for _ in range(n_prof):
            plan.contract(blocks.ptrs, res, ws, mode=0, key=1)
        torch.cuda.synchronize()
        prof = {k: (n, t_ms / n_prof) for k, (n, t_ms) in comet.profile_read().items()}
        comet.profile_enable(False)
        entry["kernels_ms"] = prof
        if prec == "split_bf16":
            k_ms = prof.get("batched_split", (1, t))[1]
            tile = info["tile"]
            # MMA work the kernel issues: K in chunks of 16, M in 128-row tiles, N in strips
            issued = sum(6 * 2.0 * (-(-int(r[3] * r[0] * r[1]) // tile[0]) * tile[0]) *
                         (-(-int(r[2] * r[4] * r[5]) // tile[1]) * tile[1]) * (-(-int(r[6]) // 16) * 16) for r in ext)
            achieved = 6 * plan.flops / (k_ms * 1e-3) / 1e12
            peak = peaks.get("bf16_tflops", 1900.0)
            entry["roofline"] = {"kernel": "batched_split (tcgen05)", "bound": "tensor", "achieved": achieved,
                                 "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                                 "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)",
                                 "achieved_counts": "6 BF16 products x 2*M*N*K per block, unpadded",
                                 "issued_mma_tflops": issued / (k_ms * 1e-3) / 1e12,
                                 "issued_frac": issued / (k_ms * 1e-3) / 1e12 / peak,
                                 "issued_counts": "6 x 2 x M rounded to 128 x N rounded to the strip x K rounded to 16",
                                 "ms_per_launch": k_ms}
            entry["prepass_ms"] = prof.get("batched_prepass", (0, 0.0))[1]
        else:
            k_ms = prof.get("batched_f64", (1, t))[1]
            entry["roofline"] = {"kernel": "batched_f64", "bound": "fp64", "achieved": plan.flops / (k_ms * 1e-3) / 1e12,
                                 "peak": fp64_peak["tflops"], "unit": "TFLOP/s",
                                 "frac": plan.flops / (k_ms * 1e-3) / 1e12 / fp64_peak["tflops"],
                                 "peak_source": "measured: " + fp64_peak["how"] + ", " + fp64_peak["probe"]}
        # CPU baseline leg: the oracle on three blocks, and the error of the GPU's (s_b, q_b)
        import oracle
        got = res.cpu().numpy().reshape(-1, 2)
        t_cpu, cfl, es, eq = 0.0, 0.0, 0.0, 0.0
        for b in check:
            A = blocks.host_operand(b, 0).astype(np.float64)
            B = blocks.host_operand(b, 1).astype(np.float64)
            t0 = time.perf_counter()
            sr, qr = oracle.triples_reduce(A, B, 1, b)
            t_cpu += time.perf_counter() - t0
            cfl += fl[b]
            n_el = float(np.prod(shapes(ext[b])[2]))
            eq = max(eq, abs(got[b, 1] - qr) / qr)
            es = max(es, abs(got[b, 0] - sr) / np.sqrt(qr * n_el))
        entry["cpu_baseline"] = {"value": cfl / t_cpu / 1e9, "unit": "GFLOP/s", "cores": oracle.threads(),
                                 "kind": "oracle", "sample": f"blocks {check} (smallest, median, largest), s_b and q_b"}
        entry["error"] = {"q_rel": eq, "s_rel_to_sqrt_qn": es, "blocks": check,
                          "tolerance": 1e-6 if prec == "split_bf16" else 1e-12}
        out[prec] = entry
        del blocks, ws, res, g
        torch.cuda.empty_cache()
    if "native" in out:
        out["split_speedup_over_fp64"] = out["native"]["ms_per_step"] / out["split_bf16"]["ms_per_step"]
    # store mode (every output element materialised): the blocks from the first whose FP32 outputs
    # fit in 64 GB, one launch; bound by the HBM writes of T
    elems = np.prod(ext[:, :6].astype(np.float64), axis=1)
    n_s = int(np.searchsorted(np.cumsum(elems) * 4, 64e9, side="right"))
    blocks = Blocks(ext[:n_s], np.float32)
    plan = comet.BatchedPlan(TEXPR, LABELS, ext[:n_s], "f32", precision="split_bf16")
    ws = plan.workspace()
    plan.prepare(ws)
    sizes = (elems[:n_s].astype(np.int64) + 3) // 4 * 4          # 16-byte aligned block starts
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    obuf = torch.empty(int(sizes.sum()), dtype=torch.float32, device="cuda")
    table = torch.tensor(offs * 4, dtype=torch.int64, device="cuda") + obuf.data_ptr()
    plan.contract(blocks.ptrs, table, ws, mode=1)
    torch.cuda.synchronize()
    comet.profile_enable(True)
    comet.profile_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(2):
        plan.contract(blocks.ptrs, table, ws, mode=1)
    e1.record()
    torch.cuda.synchronize()
    prof = comet.profile_read()
    comet.profile_enable(False)
    comet.sync_status()
    t = e0.elapsed_time(e1) / 2
    k_ms = prof.get("batched_split", (2, 2 * t))[1] / 2
    wbytes = float(elems[:n_s].sum()) * 4
    hbm = (peaks or {}).get("hbm_gbs", 6792.1)
    out["store_split_bf16"] = {"blocks": n_s, "ms_per_launch": t, "kernel_ms": k_ms, "output_bytes": wbytes,
                               "gflops": plan.flops / (t * 1e-3) / 1e9,
                               "roofline": {"bound": "hbm", "achieved": wbytes / (k_ms * 1e-3) / 1e9,
                                            "peak": hbm, "unit": "GB/s",
                                            "frac": wbytes / (k_ms * 1e-3) / 1e9 / hbm,
                                            "algorithmic_bytes": "4 B per output element written"}}
    del blocks, ws, obuf, table
    torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    return 0


def run_triples_energy(a) -> int:
    """The fused CCSD(T)-style accumulation: per block, T[a,b,c,i,j,k] = the nine permuted terms
    sign * X_p[d,..] * Y_p[..,d,..] and E_b = sum T^2 / D_b, with D the signed sum of per-label
    eps vectors; extents uniform 8..32 (the batched triples table, seed 3), operands uniform
    [-1,1) (seed 11), eps uniform in [1,2) (virtual) and [-2,-1) (occupied).  One launch per step;
    T never goes to memory.  CPU baseline leg: the oracle on the three smallest blocks (timed, and
    the error of the GPU energies against it).  Prints
    one JSON line (not the headline line)."""
    import numpy as np
    import torch
    import paper_2102_06827_gb300 as comet
    import synth
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from triples_terms import LABELS, SIGNS, T_LABELS, operand_labels, terms
    dev = torch.device("cuda", 0)
    tl = terms()
    col = {l: q for q, l in enumerate(LABELS)}
    out = {"workload": "fused triples energy: nine permuted terms per block, E_b = sum T^2/D_b; "
                       "extents uniform 8..32 (seed 3), operands uniform [-1,1) (seed 11)"}
    fp64_peak = measure_fp64_peak()

    def build(n_blocks, dtype):
        ext = synth.triples_blocks(4096)[:n_blocks]
        sizes, eps_sizes = [], []
        for b in range(n_blocks):
            for e in tl:
                for ls in operand_labels(e):
                    sizes.append(int(np.prod([ext[b, col[l]] for l in ls])))
            for l in T_LABELS:
                eps_sizes.append(int(ext[b, col[l]]))
        sizes = np.array(sizes, dtype=np.int64)
        total = int(sizes.sum())
        buf = torch.empty(total, dtype=dtype, device=dev)
        chunk = 1 << 27
        for c0 in range(0, total, chunk):
            n = min(chunk, total - c0)
            buf[c0:c0 + n] = synth.torch_uniform(11, c0 // chunk, n, dev).to(dtype)
        offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]) * buf.element_size()
        ops = torch.tensor(offs, dtype=torch.int64, device=dev) + buf.data_ptr()
        eps_sizes = np.array(eps_sizes, dtype=np.int64)
        shift = np.concatenate([np.full(n, 1.5 if q % 6 < 3 else -1.5) for q, n in enumerate(eps_sizes)])
        ebuf = (synth.torch_uniform(12, 0, int(eps_sizes.sum()), dev) * 0.5 +
                torch.from_numpy(shift).to(dev)).to(dtype)
        eoffs = np.concatenate([[0], np.cumsum(eps_sizes)[:-1]]) * ebuf.element_size()
        eps = torch.tensor(eoffs, dtype=torch.int64, device=dev) + ebuf.data_ptr()
        return ext, buf, ops, ebuf, eps, sizes, eps_sizes

    def cpu_baseline(ext, buf, ebuf, sizes, eps_sizes, energies, dtype, n_check=3):
        """the CPU baseline leg: the oracle on the three smallest blocks, timed on the host cores,
        and the relative error of the GPU energies of those blocks against it"""
        import oracle
        hb = buf  # host copies of the checked blocks only
        per_block = len(tl) * 2
        starts = np.concatenate([[0], np.cumsum(sizes)])
        estarts = np.concatenate([[0], np.cumsum(eps_sizes)])
        sel = np.argsort(np.prod(ext[:, :6], axis=1))[:n_check]
        worst, t_cpu, flops = 0.0, 0.0, 0.0
        for b in sel:
            ops = []
            for p, e in enumerate(tl):
                pair = []
                for q, ls in enumerate(operand_labels(e)):
                    k = b * per_block + 2 * p + q
                    v = hb[int(starts[k]):int(starts[k + 1])].double().cpu().numpy()
                    pair.append(np.reshape(v, [int(ext[b, col[l]]) for l in ls], order="F"))
                ops.append(tuple(pair))
            eps = [ebuf[int(estarts[b * 6 + q]):int(estarts[b * 6 + q + 1])].double().cpu().numpy()
                   for q in range(6)]
            t0 = time.perf_counter()
            ref = oracle.triples_energy(tl, ops, eps, SIGNS)[0]
            t_cpu += time.perf_counter() - t0
            flops += len(tl) * 2.0 * float(np.prod(ext[b, :7]))
            worst = max(worst, abs(float(energies[b]) - ref) / abs(ref))
        return {"value": flops / t_cpu / 1e9, "unit": "GFLOP/s", "cores": oracle.threads(), "kind": "oracle",
                "sample": f"blocks {[int(x) for x in sel]} (the smallest), whole energies",
                "max_rel_err": worst}

    for name, dtype, n_blocks, steps in (("f32", torch.float32, a.te_blocks, max(1, min(a.steps, 3))),
                                         ("f64", torch.float64, a.te_f64_blocks, 1)):
        ext, buf, ops, ebuf, eps, sizes, eps_sizes = build(n_blocks, dtype)
        plan = comet.TriplesPlan(tl, LABELS, ext, SIGNS, dtype)
        ws = plan.workspace(dev)
        plan.prepare(ws)
        en = torch.empty(n_blocks, dtype=torch.float64, device=dev)
        plan.energy(ops, eps, en, ws)   # warm-up
        comet.sync_status()
        clocks = ClockSampler(0)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            plan.energy(ops, eps, en, ws)
        e1.record()
        torch.cuda.synchronize()
        ck = clocks.stop() or {}
        comet.sync_status()
        t = e0.elapsed_time(e1) / steps
        energies = en.cpu().numpy()
        sm_mhz = ck.get("sm_mhz") or 1900.0
        # FMA pipe peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flops per clock (FP64:
        # the measured FP64 probe peak); the kernel's useful flops are plan.flops
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12 if name == "f32" else fp64_peak["tflops"]
        achieved = plan.flops / (t * 1e-3) / 1e12
        roof = {"bound": "alu" if name == "f32" else "fp64", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": ("FP32 FMA lanes x median SM clock under load" if name == "f32"
                                else "measured: " + fp64_peak["how"] + ", " + fp64_peak["probe"])}
        if name == "f32" and plan.info.get("tensor_core"):
            # the tensor-core path: six BF16 products of 128 x 64 per pair-tile (8 x 4^5 of T), term
            # and 16 summed indices (the summed label rounded up to 16), against the BF16 burst peak;
            # the useful flops against the FP32 FMA rate stay beside it
            e64 = ext.astype(np.int64)
            pt = -(-e64[:, col["a"]] // 8)
            for l in "bcijk":
                pt = pt * -(-e64[:, col[l]] // 4)
            mma_flops = float(np.sum(pt * len(tl) * 6 * 2 * 128 * 64 * 16 * -(-e64[:, col["d"]] // 16)))
            peaks = measured_peaks() or {}
            bpk = peaks.get("bf16_tflops", 1900.0)
            issued = mma_flops / (t * 1e-3) / 1e12
            # the bound the design identifies: shared-memory bytes per pair-tile, modelled from the
            # kernel's data flow (TMA fills of both operands' three planes per 32 summed indices;
            # MMA operand reads of 128 + 64 rows x 32 bytes per product and 16 indices; the
            # drain's read and write of the 32 KB pair-tile per term, the first term a write only;
            # the energy pass's read), against 128 bytes per clock per SM at the sampled clock
            ed = e64[:, col["d"]]
            nt = len(tl)
            per_pt = (nt * (-(-ed // 32) * 3 * (128 + 64) * 64 + -(-ed // 16) * 6 * (128 + 64) * 32)
                      + 32768 + (nt - 1) * 65536 + 32768)
            smem_bytes = float(np.sum(pt * per_pt))
            smem_peak = 152 * 128 * sm_mhz * 1e6 / 1e12
            smem_tbs = smem_bytes / (t * 1e-3) / 1e12
            roof = {"bound": "tensor", "achieved": issued, "peak": bpk, "unit": "TFLOP/s", "frac": issued / bpk,
                    "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)",
                    "mma_flops_issued": mma_flops, "pair_tiles": int(plan.info["pair_tiles"]),
                    "useful_vs_fp32_fma": {"achieved": achieved, "peak": peak, "frac": achieved / peak,
                                           "peak_source": "FP32 FMA lanes x median SM clock under load"},
                    "shared_memory_model": {"bytes": smem_bytes, "bytes_per_pair_tile": smem_bytes / float(np.sum(pt)),
                                            "achieved": smem_tbs, "peak": smem_peak, "unit": "TB/s",
                                            "frac": smem_tbs / smem_peak,
                                            "peak_source": "152 SMs x 128 bytes per clock x median SM clock"}}
        out[name] = {"blocks": n_blocks, "ms_per_step": t, "steps": steps, "tflops": achieved,
                     "roofline": roof, "path": ("tensor cores (split BF16, 6 products)"
                                                if name == "f32" and plan.info.get("tensor_core") else "FMA"),
                     "tiles": plan.info["tiles"], "flops": plan.flops, "clocks": ck,
                     "energy_sum": float(energies.sum()),
                     "cpu_baseline": cpu_baseline(ext, buf, ebuf, sizes, eps_sizes, energies, dtype)}
        del buf, ebuf, ops, eps, ws, en
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    return 0


def run_small_and_chain(a) -> int:
    """The extent-24 FP64 contraction (plus its bit-exact transpose) and the differentiated
    three-operand chain (forward + backward through the autograd function, split-BF16 on FP32
    storage).  Prints one JSON line (not the headline line)."""
    import torch
    import paper_2102_06827_gb300 as comet
    from paper_2102_06827_gb300 import autograd
    import synth
    dev = torch.device("cuda", 0)
    out = {}
    # extent-24 FP64 contraction, timed as a captured graph of 100 launches
    e24 = "C[a,b,c,d] = A[a,e,b] * B[e,d,c]"
    ext = dict(a=24, b=24, c=24, d=24, e=24)
    p = comet.Plan(e24, ext, torch.float64)
    A = synth.torch_uniform(0, 0, 24 ** 3, dev)
    B = synth.torch_uniform(0, 1, 24 ** 3, dev)
    C = torch.empty(24 ** 4, dtype=torch.float64, device=dev)
    T = torch.empty_like(A)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p.contract([A, B], C, stream=s)
        comet.transpose(A, (24, 24, 24), (2, 0, 1), out=T, stream=s)
    torch.cuda.synchronize()
    for name, fn in (("contract", lambda: p.contract([A, B], C, stream=s)),
                     ("transpose", lambda: comet.transpose(A, (24, 24, 24), (2, 0, 1), out=T, stream=s))):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(100):
                fn()
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / 1000 * 1e3
        out["extent24_" + name + "_us"] = us
    out["extent24_contract_gflops"] = p.flops / (out["extent24_contract_us"] * 1e-6) / 1e9
    out["extent24_transpose_gbs"] = 2 * 8 * 24 ** 3 / (out["extent24_transpose_us"] * 1e-6) / 1e9
    # differentiated chain D[a,b] = A[a,i,j] B[i,j,k,l] C[k,l,b], split-BF16 on FP32 storage
    ec = "D[a,b] = A[a,i,j] * B[i,j,k,l] * C[k,l,b]"
    shapes = [(256, 48, 48), (48, 48, 48, 48), (48, 48, 256)]
    xs = [synth.torch_uniform(4, t, math.prod(sh), dev, dtype=torch.float32).view(tuple(reversed(sh)))
          .requires_grad_(True) for t, sh in enumerate(shapes)]
    G = synth.torch_uniform(4, 9, 256 * 256, dev, dtype=torch.float32).view(256, 256)

    def step():
        for x in xs:
            x.grad = None
        D = autograd.einsum(ec, *xs, precision="split_bf16", layout="col")
        D.backward(G)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 10
    pf = comet.Plan(ec, dict(a=256, b=256, i=48, j=48, k=48, l=48), torch.float32, precision="split_bf16")
    bwd = sum(comet.Plan(autograd.adjoint_expr(ec, q), dict(a=256, b=256, i=48, j=48, k=48, l=48),
                         torch.float32, precision="split_bf16").flops for q in range(3))
    out["chain_fwd_bwd_ms"] = ms
    out["chain_flops_fwd"] = pf.flops
    out["chain_flops_bwd"] = bwd
    out["chain_gflops"] = (pf.flops + bwd) / (ms * 1e-3) / 1e9
    out["chain_order"] = pf.info["order"]
    comet.sync_status()
    print(json.dumps(out), flush=True)
    return 0


def _time_plan(plan, ins, out, ws, reps=5, graph=False):
    """ms per contraction: eager launches, or one captured CUDA graph of `reps` contractions
    (which removes the host launch cost that dominates small multi-step plans)."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    for _ in range(2):
        plan.contract(ins, out, ws, stream=s)
    g = None
    if graph:
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(reps):
                plan.contract(ins, out, ws, stream=s)
        with torch.cuda.stream(s):
            g.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):  # CUDAGraph.replay() launches on the current stream
        e0.record(s)
        if g is not None:
            g.replay()
        else:
            for _ in range(reps):
                plan.contract(ins, out, ws, stream=s)
        e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_ablation(a) -> int:
    """The paper's two ablations on this GPU (split-BF16 path, FP32 storage):
    (1) the multi-operand expressions of Table 1, natural left-to-right order vs the planned
        order, occupied labels i,j,m,n = o and virtual labels a..f = v for (o, v) = (24, 72)
        and (64, 192), synthetic extents, timed eagerly and as one captured CUDA graph;
    (2) every enumerated TTGT form of two contractions vs the planner's choice (best vs
        arbitrary permutation).  Prints one JSON line."""
    import re
    import torch
    import paper_2102_06827_gb300 as comet
    import synth
    dev = torch.device("cuda", 0)
    out = {"table1": [], "forms": []}
    rows = [l.split("|") for l in open(os.path.join(ROOT, "tests", "golden", "table1_expressions.txt"))
            if l.strip() and not l.startswith("#")]
    for (o_ext, v_ext) in ((24, 72), (64, 192)):
        for rhs, paper in rows:
            ops = [[x.strip() for x in t.split(",")] for t in re.findall(r"\[([^\]]*)\]", rhs)]
            cnt = {}
            for o in ops:
                for l in o:
                    cnt[l] = cnt.get(l, 0) + 1
            outl = [l for o in ops for l in o if cnt[l] == 1]
            ext = {l: (o_ext if l in "ijmn" else v_ext) for o in ops for l in o}
            expr = f"X[{','.join(outl)}] = {rhs.strip()}"
            ins = [synth.torch_uniform(7, t, math.prod(ext[l] for l in o), dev, dtype=torch.float32,
                                       scale=1.0 / math.sqrt(math.prod(ext[l] for l in o)))
                   for t, o in enumerate(ops)]
            res = {"expr": expr, "o": o_ext, "v": v_ext, "paper_speedup": float(paper)}
            for order in ("planned", "natural"):
                p = comet.Plan(expr, ext, torch.float32, precision="split_bf16", order=order)
                C = torch.empty(math.prod(ext[l] for l in outl), dtype=torch.float32, device=dev)
                ws = p.workspace(dev)
                res[order + "_ms"] = _time_plan(p, ins, C, ws)
                res[order + "_graph_ms"] = _time_plan(p, ins, C, ws, graph=True)
                comet.profile_enable(True)
                comet.profile_read()
                for _ in range(3):
                    p.contract(ins, C, ws)
                torch.cuda.synchronize()
                res[order + "_kernels_ms"] = {k: (n / 3, t / 3) for k, (n, t) in comet.profile_read().items()}
                comet.profile_enable(False)
                res[order + "_flops"] = p.flops
                res[order + "_tree"] = p.info["order"]
                del ws, C
            res["speedup"] = res["natural_ms"] / res["planned_ms"]
            res["speedup_graph"] = res["natural_graph_ms"] / res["planned_graph_ms"]
            res["flop_ratio"] = res["natural_flops"] / res["planned_flops"]
            out["table1"].append(res)
            del ins
            torch.cuda.empty_cache()
    cases = [("C[i,a,j,b] = A[k,a,c,i] * B[c,b,k,j]", dict(i=48, j=48, k=48, a=144, b=144, c=144)),
             ("C[a,b,c,d] = A[a,e,b,f] * B[d,f,c,e]", dict(a=96, b=96, c=96, d=96, e=48, f=48))]
    for expr, ext in cases:
        p0 = comet.Plan(expr, ext, torch.float32, precision="split_bf16")
        n = p0.info["steps"][0]["n_forms"]
        tens = re.findall(r"\w+\[([^\]]*)\]", expr)
        outl, ins_l = tens[0], tens[1:]
        ins = [synth.torch_uniform(8, t, math.prod(ext[l.strip()] for l in o.split(",")), dev, dtype=torch.float32)
               for t, o in enumerate(ins_l)]
        C = torch.empty(math.prod(ext[l.strip()] for l in outl.split(",")), dtype=torch.float32, device=dev)
        times = []
        for k in range(n):
            p = comet.Plan(expr, ext, torch.float32, precision="split_bf16", form=k)
            ws = p.workspace(dev)
            times.append(_time_plan(p, ins, C, ws, reps=3, graph=True))
            del ws
        chosen = p0.info["steps"][0]["form_index"]
        srt = sorted(times)
        out["forms"].append({"expr": expr, "n_forms": n, "chosen": chosen, "chosen_ms": times[chosen],
                             "best_ms": srt[0], "median_ms": srt[len(srt) // 2], "worst_ms": srt[-1],
                             "best_over_worst": srt[-1] / srt[0],
                             "chosen_vs_best": times[chosen] / srt[0],
                             "chosen_over_median_speedup": srt[len(srt) // 2] / times[chosen]})
        torch.cuda.empty_cache()
    comet.sync_status()
    print(json.dumps(out), flush=True)
    return 0


def run_profile_case(case: str, a=None) -> int:
    """Small cases for ncu captures: inputs above the 129 MB L2, a few GB on the device."""
    import torch
    import paper_2102_06827_gb300 as comet
    import synth
    dev = torch.device("cuda", 0)
    if case == "gemv":   # the two tensor-times-vector steps of Table 1 row 1 at o=64 v=192 (FP32, split)
        e = "X[i,a] = A[c,d,m,n] * B[i,n,a,d] * C[m,c]"
        ext = dict(c=192, d=192, m=64, n=64, i=64, a=192)
        ops = [("c", "d", "m", "n"), ("i", "n", "a", "d"), ("m", "c")]
        ins = [synth.torch_uniform(7, t, math.prod(ext[l] for l in o), dev, dtype=torch.float32)
               for t, o in enumerate(ops)]
        plan = comet.Plan(e, ext, torch.float32, precision="split_bf16")
        X = torch.empty(64 * 192, dtype=torch.float32, device=dev)
        ws = plan.workspace(dev)
        for _ in range(2):
            plan.contract(ins, X, ws)
        comet.sync_status()
        print(json.dumps({"case": case, "steps": [s["kernel"] for s in plan.info["steps"]],
                          "large_operand_bytes": 4 * 192 * 192 * 64 * 64}))
        return 0
    if case == "triples":   # 512 of the 4096 triples blocks (same extent generator), split, reduce mode
        import numpy as np
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from batched_data import EXPR as TEXPR, LABELS, Blocks
        ext = synth.triples_blocks(512)
        blocks = Blocks(ext, np.float32)
        plan = comet.BatchedPlan(TEXPR, LABELS, ext, "f32", precision="split_bf16", tile=a.pc_tile)
        ws = plan.workspace()
        plan.prepare(ws)
        res = torch.zeros(2 * blocks.n, dtype=torch.float64, device="cuda")
        for _ in range(2):
            plan.contract(blocks.ptrs, res, ws, mode=0, key=1)
        comet.sync_status()
        print(json.dumps({"case": case, "blocks": 512, "flops": plan.flops, "tile": plan.describe()["tile"]}))
        return 0
    if case == "transpose":
        ext = tuple(int(e) for e in a.pc_extents.split(","))
        perm = tuple(int(q) for q in a.pc_perm.split(","))
        n = math.prod(ext)
        x = synth.torch_uniform(5, 0, n, dev, dtype=torch.float32 if a.pc_dtype == "f32" else torch.float64)
        y = torch.empty_like(x)
        for _ in range(2):
            comet.transpose(x, ext, perm, out=y)
        comet.sync_status()
        print(json.dumps({"case": case, "extents": ext, "perm": perm, "bytes": 2 * x.element_size() * n}))
        return 0
    o, v = (48, 160) if case in ("split", "emu") else (16, 48)
    if a is not None and a.pc_o > 0 and a.pc_v > 0:   # e.g. the headline size o=64 v=192
        o, v = a.pc_o, a.pc_v
    ext = dict(i=o, j=o, k=o, a=v, b=v, c=v)
    n = o * v * v * o
    dt = torch.float32 if case == "split" else torch.float64
    plan = comet.Plan(EXPR, ext, dt, precision={"split": "split_bf16", "emu": "emu_f64"}.get(case, "native"))
    A = synth.torch_uniform(1, 0, n, dev, dtype=dt, scale=1.0 / math.sqrt(o * v))
    B = synth.torch_uniform(2, 0, n, dev, dtype=dt, scale=1.0 / math.sqrt(o * v))
    C = torch.empty(n, dtype=dt, device=dev)
    ws = plan.workspace(dev)
    for _ in range(2):
        plan.contract([A, B], C, ws)
    comet.sync_status()
    print(json.dumps({"case": case, "extents": ext, "flops": plan.flops, "workspace": plan.workspace_bytes}))
    return 0


def config(precision="split_bf16"):
    return {"workload": WORKLOAD, "o": 64, "v": 192, "precision": precision,
            "input": "uniform[-1,1]/sqrt(64*192), SplitMix64 seeds 1 (A) and 2 (B)",
            "storage": "FP32 column-major (split path), FP64 (FP64 form)",
            "l2": "inputs (576 MiB each) larger than the 129 MB L2; no flush needed"}


# ---- clocks during the timed region ---------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---- helpers -----------------------------------------------------------------------------------
def source_hash(*paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(name: str, src_hash: str):
    """dram bytes per launch from a committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", f"{name}.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("source_hash") != src_hash:
        return None
    return d.get("dram_bytes_per_launch")


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def make_inputs(torch, dtype, device):
    import synth
    A = synth.torch_uniform(1, 0, N_ELEM, device, dtype=dtype, scale=SCALE)
    B = synth.torch_uniform(2, 0, N_ELEM, device, dtype=dtype, scale=SCALE)
    return A, B


def sample_indices(n):
    import numpy as np
    import synth
    return np.unique(synth.integers(11, 0, n, 0, N_ELEM - 1).astype(np.int64))


# ---- the reference arm: the CPU oracle ------------------------------------------------------
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    import synth
    A = synth.tensor((64, 192, 192, 64), 1, 0, scale=SCALE, dtype=np.float32).astype(np.float64)
    B = synth.tensor((192, 192, 64, 64), 2, 0, scale=SCALE, dtype=np.float32).astype(np.float64)
    sel = sample_indices(256)
    t0 = time.perf_counter()
    oracle.einsum_sampled(EXPR, A, B, sel=sel)
    dt = time.perf_counter() - t0
    n = int(min(200000, max(64, len(sel) * (6.0 / max(dt, 1e-3)))))   # ~6 s of CPU work per step
    sel = sample_indices(n)
    flops_step = 2.0 * 64 * 192 * len(sel)
    for _ in range(a.warmup):
        oracle.einsum_sampled(EXPR, A, B, sel=sel[: max(1, len(sel) // 8)])
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.einsum_sampled(EXPR, A, B, sel=sel)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = flops_step * a.steps / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(config("fp64_oracle"), sample=f"{len(sel)} outputs per step"),
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"{len(sel)} sampled outputs of C (each a 12288-term FP64 sum)"},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- replicas: one process per GPU, no collective on the data path ---------------------------
class Replicas:
    """The rank layout of a torchrun launch (RANK / LOCAL_RANK / WORLD_SIZE): every rank runs its
    own copy of the workload; the job's time is the slowest rank's (max over ranks) and its value
    all ranks' work over that time.  backend: "nccl" on GPUs, "gloo" in the CPU tests."""

    def __init__(self, backend: str, device=None):
        import torch.distributed as dist
        self.dist = dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device
        if self.world > 1 and not dist.is_initialized():
            dist.init_process_group(backend)

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.world == 1:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def throughput(self, units_per_rank: float, seconds: float) -> float:
        """whole-job units per second: every rank's units over the slowest rank's time"""
        return self.world * units_per_rank / self.max(seconds)

    def close(self):
        if self.world > 1 and self.dist.is_initialized():
            self.dist.destroy_process_group()


# ---- our arm -------------------------------------------------------------------------------------
def main():
    a = args_parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.profile_case:
        return run_profile_case(a.profile_case, a)
    if a.sweep == "transpose":
        return run_transpose_sweep()
    if a.peak == "fp64":
        return run_peak_fp64(a)
    if a.workload == "triples":
        return run_triples(a)
    if a.workload == "small":
        return run_small_and_chain(a)
    if a.workload == "triples_energy":
        return run_triples_energy(a)
    if a.ablation:
        return run_ablation(a)
    import numpy as np
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    reps = Replicas("nccl", dev)
    world, rank = reps.world, reps.rank
    import paper_2102_06827_gb300 as comet
    barrier = reps.barrier
    max_over_ranks = reps.max

    stream = torch.cuda.current_stream()
    # ---------------- split-BF16 path (the headline) ----------------
    plan = comet.Plan(EXPR, EXT, torch.float32, precision="split_bf16")
    flops = plan.flops
    A, B = make_inputs(torch, torch.float32, dev)
    C = torch.empty(N_ELEM, dtype=torch.float32, device=dev)
    ws = plan.workspace(dev)
    for _ in range(a.warmup):
        plan.contract([A, B], C, ws)
    comet.sync_status()
    barrier()
    torch.cuda.synchronize()
    comet.profile_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        plan.contract([A, B], C, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    prof = comet.profile_read()
    comet.profile_enable(False)
    comet.sync_status()
    ms_total = max_over_ranks(e0.elapsed_time(e1))
    ms_step = ms_total / a.steps
    value = world * flops * a.steps / (ms_total * 1e-3) / 1e9
    # kernels, not profiler scopes: a split GEMM scope launches the whole-K kernel, and with a
    # stream-K tail the K-sliced kernel and its reduce as well (with K slices throughout: the
    # sliced kernel and the reduce)
    st0 = plan.info["steps"][0]
    per_gemm = 3 if st0.get("tail_slices", 1) > 1 else 2 if st0.get("ksplit", 1) > 1 else 1
    launches = sum(v[0] for k, v in prof.items()) + (per_gemm - 1) * prof.get("gemm_split_bf16", (0, 0.0))[0]
    g_launch, g_ms = prof.get("gemm_split_bf16", (0, 0.0))
    p_launch, p_ms = prof.get("split_prepass", (0, 0.0))
    gemm_ms = g_ms / max(1, g_launch)
    peaks = measured_peaks()
    peak_src = "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    peak = peaks.get("bf16_tflops") if peaks else None
    if not peak:
        peak, peak_src = 1900.0, "fallback (recipe, burst)"
    achieved = 6.0 * flops / (gemm_ms * 1e-3) / 1e12
    src = source_hash("paper_2102_06827_gb300/csrc/k_gemm_split.cu", "paper_2102_06827_gb300/csrc/sm100.cuh")
    traffic = recorded_traffic("gemm_split_bf16_ccsd", src)
    pre_bytes = 2.0 * N_ELEM * (4 + 6)
    roofline = {"kernel": "gemm_split_bf16", "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": peak_src,
                "peak_sustained": peaks.get("bf16_tflops_sustained") if peaks else None,
                "frac_of_sustained": achieved / peaks["bf16_tflops_sustained"] if peaks else None,
                "achieved_counts": "6 BF16 products x 2*M*N*K per GEMM (M=N=K=12288)",
                "gemm_launches": (f"{st0.get('tail_tiles', 0)} tail tiles in {st0.get('tail_slices', 1)} K slices "
                                  "after the whole-K waves, then the reduce" if st0.get("tail_slices", 1) > 1
                                  else "one whole-K launch"),
                "ms_per_launch": gemm_ms,
                "effective_fp32_tflops": flops / (gemm_ms * 1e-3) / 1e12}
    # the cuBLAS peak was taken at its own clocks: time x SM clock makes the two comparable
    peak_mhz = ((peaks or {}).get("clocks_under_load") or {}).get("sm_mhz_median")
    run_mhz = (clk or {}).get("sm_mhz")
    if peak_mhz and run_mhz:
        roofline["clock_normalised"] = {
            "sm_mhz_this_run": run_mhz, "sm_mhz_of_peak_measurement": peak_mhz,
            "frac_at_equal_clock": achieved / peak * peak_mhz / run_mhz,
            "note": "frac x (peak's median SM clock / this run's median SM clock): the work per clock "
                    "against cuBLAS's"}
    prepass = {"kernel": "split_prepass", "launches_per_step": p_launch / max(1, a.steps),
               "ms_per_step": p_ms / max(1, a.steps), "bytes_per_step": pre_bytes,
               "achieved_gbs": pre_bytes / (p_ms / max(1, a.steps) * 1e-3) / 1e9 if p_ms else None,
               "peak_gbs": peaks.get("hbm_gbs") if peaks else 6800.0}
    prepass["frac"] = prepass["achieved_gbs"] / prepass["peak_gbs"] if prepass["achieved_gbs"] else None
    # the same time against every byte the pass moves: the abs-max launch reads both operands once
    # more before the split can start (the fixed-point grid needs each operand's largest magnitude)
    moved = pre_bytes + 2.0 * N_ELEM * 4
    prepass["bytes_moved_per_step"] = moved
    prepass["frac_of_bytes_moved"] = (moved / (p_ms / max(1, a.steps) * 1e-3) / 1e9 / prepass["peak_gbs"]
                                      if p_ms else None)

    # ---------------- FP64 form of the same contraction ----------------
    plan64 = comet.Plan(EXPR, EXT, torch.float64, precision="native")
    # genuine FP64 operands (53-bit uniforms of the same seeds), not FP32 data widened: the
    # products then round in FP64 and the stated FP64 error means something
    A64, B64 = make_inputs(torch, torch.float64, dev)
    C64 = torch.empty(N_ELEM, dtype=torch.float64, device=dev)
    plan64.contract([A64, B64], C64)
    comet.sync_status()
    barrier()
    comet.profile_enable(True)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(a.fp64_steps):
        plan64.contract([A64, B64], C64)
    f1.record(stream)
    torch.cuda.synchronize()
    prof64 = comet.profile_read()
    comet.profile_enable(False)
    comet.sync_status()
    ms64 = max_over_ranks(f0.elapsed_time(f1)) / a.fp64_steps
    gflops64 = world * flops / (ms64 * 1e-3) / 1e9
    k64 = prof64.get("gemm_f64", (1, ms64))
    fp64_peak = measure_fp64_peak()
    fp64 = {"gflops": gflops64, "ms_per_step": ms64, "steps": a.fp64_steps,
            "roofline": {"kernel": "gemm_f64", "bound": "fp64", "achieved": flops / (k64[1] / k64[0] * 1e-3) / 1e12,
                         "peak": fp64_peak["tflops"], "unit": "TFLOP/s",
                         "frac": flops / (k64[1] / k64[0] * 1e-3) / 1e12 / fp64_peak["tflops"],
                         "peak_source": "measured in this run: " + fp64_peak["how"] + ", fastest probe "
                                        + fp64_peak["probe"],
                         "probes_tflops": fp64_peak["probes_tflops"]},
            "split_speedup_over_fp64": ms64 / ms_step}

    # ---------------- the same FP64 contraction emulated on the BF16 tensor cores ----------------
    plan_e = comet.Plan(EXPR, EXT, torch.float64, precision="emu_f64")
    ws_e = plan_e.workspace(dev)
    Ce = torch.empty(N_ELEM, dtype=torch.float64, device=dev)
    for _ in range(2):
        plan_e.contract([A64, B64], Ce, ws_e)
    comet.sync_status()
    barrier()
    comet.profile_enable(True)
    comet.profile_read()
    f0.record(stream)
    for _ in range(a.emu_steps):
        plan_e.contract([A64, B64], Ce, ws_e)
    f1.record(stream)
    torch.cuda.synchronize()
    prof_e = comet.profile_read()
    comet.profile_enable(False)
    comet.sync_status()
    ms_e = max_over_ranks(f0.elapsed_time(f1)) / a.emu_steps
    ke = prof_e.get("gemm_emu_bf16x6", (1, ms_e))
    pe = prof_e.get("split_prepass", (0, 0.0))
    emu_gemm_ms = ke[1] / max(1, ke[0])
    emu_achieved = 21.0 * flops / (emu_gemm_ms * 1e-3) / 1e12
    fp64["emulated"] = {
        "precision": "emu_f64 (six bf16 slices, 21 products, exact chunk sums folded into int64)",
        "gflops": world * flops / (ms_e * 1e-3) / 1e9, "ms_per_step": ms_e, "steps": a.emu_steps,
        "prepass_ms_per_step": pe[1] / max(1, a.emu_steps),
        "roofline": {"kernel": "gemm_emu_bf16x6", "bound": "tensor", "achieved": emu_achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": emu_achieved / peak, "peak_source": peak_src,
                     "achieved_counts": "21 BF16 products x 2*M*N*K per launch", "ms_per_launch": emu_gemm_ms},
        "speedup_over_native_fp64": ms64 / ms_e}
    del ws_e

    # ---------------- end to end through the C ABI with host buffers ----------------
    hA = torch.empty(N_ELEM, dtype=torch.float32, pin_memory=True)
    hB = torch.empty(N_ELEM, dtype=torch.float32, pin_memory=True)
    hC = torch.empty(N_ELEM, dtype=torch.float32, pin_memory=True)
    hA.copy_(A)
    hB.copy_(B)
    dA, dB, dC = torch.empty_like(A), torch.empty_like(B), torch.empty_like(C)
    plan.contract_host([hA, hB], hC, [dA, dB], dC, ws)
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.e2e_steps):
        plan.contract_host([hA, hB], hC, [dA, dB], dC, ws)
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    # the host result against the device result of the timed steps (the slices take their own
    # operand scales, so the two agree to the split path's error, not bitwise)
    e2e_diff = float((hC.to(dev) - C).abs().max() / C.abs().max())
    # the same call with the slice pipeline switched off (copies, contraction, copy back in order)
    plan_serial = comet.Plan(EXPR, EXT, torch.float32, precision="split_bf16", host_slices=1)
    plan_serial.contract_host([hA, hB], hC, [dA, dB], dC, ws)
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.e2e_steps):
        plan_serial.contract_host([hA, hB], hC, [dA, dB], dC, ws)
    t_serial = max_over_ranks(time.perf_counter() - t0)
    plan_serial.close()
    # K evaluations in one comet_contract_host_n call: every evaluation copies its inputs from
    # pinned host memory and its result back (alternating between two host result buffers), and
    # the copies of evaluation t + 1 overlap the GEMMs of evaluation t
    plan.contract_host([hA, hB], hC, [dA, dB], dC, ws)
    single_ref = hC.clone()
    hC2 = torch.empty(N_ELEM, dtype=torch.float32, pin_memory=True)
    outs = [hC if t % 2 == 0 else hC2 for t in range(a.steps)]
    plan.contract_host_n([[hA, hB]] * max(2, min(a.warmup, 3)), outs[:max(2, min(a.warmup, 3))], [dA, dB], dC, ws)
    barrier()
    t0 = time.perf_counter()
    plan.contract_host_n([[hA, hB]] * a.steps, outs, [dA, dB], dC, ws)
    t_pipe = max_over_ranks(time.perf_counter() - t0)
    pipe_equal = bool(torch.equal(hC, single_ref) and (a.steps < 2 or torch.equal(hC2, single_ref)))
    del hC2, outs
    e2e = {"value": world * flops * a.steps / t_pipe / 1e9, "unit": "GFLOP/s",
           "h2d_bytes_per_step": 2 * N_ELEM * 4, "d2h_bytes_per_step": N_ELEM * 4,
           "steps": a.steps, "ms_per_step": 1e3 * t_pipe / a.steps,
           "api": "comet_contract_host_n: K evaluations from pinned host buffers in one call, each "
                  "copying its inputs in and its result back inside the timed region; the copies of "
                  "one evaluation overlap the GEMMs of the one before (wall clock around the call)",
           "results_equal_single_calls": pipe_equal,
           "host_pipe": plan.info.get("host_pipe"), "max_rel_diff_vs_device": e2e_diff,
           "single_call": {"api": "comet_contract_host, one synchronising call per evaluation",
                           "value": world * flops * a.e2e_steps / t_e2e / 1e9, "steps": a.e2e_steps,
                           "ms_per_step": 1e3 * t_e2e / a.e2e_steps},
           "serial_value": world * flops * a.e2e_steps / t_serial / 1e9,
           "serial_ms_per_step": 1e3 * t_serial / a.e2e_steps}

    # ---------------- CPU baseline (oracle) and the stated error ----------------
    cpu, err = None, None
    if rank == 0 and not a.no_cpu_baseline:
        import oracle
        hA64 = np.asfortranarray(hA.numpy().astype(np.float64).reshape((64, 192, 192, 64), order="F"))
        hB64 = np.asfortranarray(hB.numpy().astype(np.float64).reshape((192, 192, 64, 64), order="F"))
        sel = sample_indices(128)
        t0 = time.perf_counter()
        oracle.einsum_sampled(EXPR, hA64, hB64, sel=sel)
        dt = time.perf_counter() - t0
        n = int(min(400000, max(128, len(sel) * a.cpu_seconds / max(dt, 1e-3))))
        sel = sample_indices(n)
        t0 = time.perf_counter()
        ref = oracle.einsum_sampled(EXPR, hA64, hB64, sel=sel)
        t_cpu = time.perf_counter() - t0
        cflops = 2.0 * 64 * 192 * len(sel)
        cpu = {"value": cflops / t_cpu / 1e9, "unit": "GFLOP/s", "cores": oracle.threads(), "kind": "oracle",
               "sample": f"{len(sel)} sampled outputs of C (each a 12288-term FP64 sum), {t_cpu:.1f} s"}
        # the FP64 forms ran on genuine FP64 operands: their reference is the oracle on those
        del hA64, hB64
        gA64 = np.asfortranarray(A64.cpu().numpy().reshape((64, 192, 192, 64), order="F"))
        gB64 = np.asfortranarray(B64.cpu().numpy().reshape((192, 192, 64, 64), order="F"))
        ref64 = oracle.einsum_sampled(EXPR, gA64, gB64, sel=sel)
        del gA64, gB64
        got = C.cpu().numpy().astype(np.float64)[sel]
        got64 = C64.cpu().numpy()[sel]
        got_e = Ce.cpu().numpy()[sel]
        den, den64 = float(np.abs(ref).max()), float(np.abs(ref64).max())

        def e_of(x, r, d, tol, inputs):
            return {"normwise_rel": float(np.abs(x - r).max() / d), "max_abs": float(np.abs(x - r).max()),
                    "tolerance": tol, "inputs": inputs}
        err = {"split_bf16": e_of(got, ref, den, 1e-6, "FP32 uniforms"),
               "fp64": e_of(got64, ref64, den64, 1e-12, "FP64 uniforms (53-bit)"),
               "emu_f64": e_of(got_e, ref64, den64, 1e-12, "FP64 uniforms (53-bit)"),
               "samples": len(sel)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16", "data": "synthetic", "config": config(),
                "roofline": roofline, "prepass": prepass, "fp64": fp64, "error": err, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "dtype_note": "bf16 x bf16 tensor-core products of a 3-way split, fp32 accumulation"}
        print(json.dumps(line), flush=True)
    reps.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
