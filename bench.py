"""Benchmark: fragment CCSD(T) on one diamond-like fragment (nocc=16, nvir=240, naux=960), mixed precision.

A step is one pass of the whole per-fragment hot path through the C-ABI: integral assembly
(lnocc_build_ints), the CCSD solve (lnocc_ccsd), the projected CCSD/MP2 fragment energies
(lnocc_fragment_energy) and the projected (T) energy (lnocc_triples), on synthetic inputs that stand
in for the paper's diamond fragment (seeded generator in paper_2407_11258_gb300/synth.py).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-fp64] [--no-cpu]
                    [--extras all|none]
    python bench.py --workload batch [--nfrag 128] [--workers 0] [--autotune 1] [--steps 1] [--warmup 1]
    python bench.py --workload mlp [--ntrain 2000] [--nheld 256] [--train-steps 2000] [--mlp-precision mixed]
    python bench.py --workload triples      # nocc=32, nvir=480, naux=1600: one solve, (T) timed, plus the
                                            # scaled fragment's error against the stored oracle energies
    python bench.py --workload case --nocc 16 --nvir 120 --naux 480 --iters 4 [--fp64] [--mlp-guess]
                                            # one solve with the library's timings printed (profiling runs)

Prints one JSON line (rank 0). `value` is model TFLOP/s of whole solves with inputs resident in HBM
(inputs of 0.5 GB exceed the 129 MB L2, so no flush is needed between steps); `e2e` repeats the
measurement with the inputs in pinned host memory, copied in every step, and the energies read back.
Multi-GPU runs shard independent fragments (one per rank per step) with no collective in the data path.
By default the line also carries `extras`: the first 16 fragments of the uneven batch, the (T)-dominated
fragment and the learned guess at its stated size (2000 training solves, 256 held out), measured after
the timed region (`--extras none` skips them).

`--workload batch` instead times whole batches of uneven fragments (nocc U{8..24}, nvir U{120..360},
naux = 4 nvir, half small-gap) through lnocc_solve_batch: a step is one batch, `value` its model
TFLOP/s and `solves_per_s` fragments per second; with N ranks the one list is split by LPT. `--workload mlp` trains the learned T2 guess on GPU
solves and reports held-out CCSD iteration counts and times from the MP2 and the learned guess.
"""
from __future__ import annotations

import argparse
import contextlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fragment CCSD(T) TFLOP/s & solves/s, mixed vs FP64 GPU at |dE|<=1e-6 Eh"
WORKLOAD = "diamond_like nocc=16 nvir=240 naux=960 projector=2 LMOs"


def model_flops(o, v, n_iter):
    """Work model: CCSD 2o^2v^4 + 16o^3v^3 + 2o^4v^2 per iteration, (T) 6o^3v^4 + 6o^4v^3, assembly 2N(...)."""
    ccsd = (2 * o**2 * v**4 + 16 * o**3 * v**3 + 2 * o**4 * v**2) * n_iter
    trip = 6 * o**3 * v**4 + 6 * o**4 * v**3
    return ccsd, trip


def triples_algorithmic_flops(o, v):
    """Contraction flops the (T) kernels execute per call: every sorted virtual triple once (2o^3v^4 + 2o^4v^3)."""
    return 2.0 * o**3 * v**4 + 2.0 * o**4 * v**3


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("bf16_tflops"), d.get("bf16_tflops_sustained"), d.get("hbm_gbs"), "measured"
    return 1900.0, 1700.0, 6800.0, "fallback"


TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_gemm_tc_triples_traffic_nocc16_nvir240.md")
TRAFFIC_SOURCES = ("paper_2407_11258_gb300/csrc/gemm.cu", "paper_2407_11258_gb300/csrc/triples.cu")


def sources_digest():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes (read + write) of the (T) contraction launches of one lnocc_triples call, from the ncu
    summary under profiles/, or None when the kernel sources have changed since that capture (the summary
    records a digest of them)."""
    if not os.path.exists(TRAFFIC_PROFILE):
        return None, "no capture"
    rec = {}
    for line in open(TRAFFIC_PROFILE):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            rec[k.strip()] = v.strip().strip("`")
    try:
        tb, dig = float(rec["traffic_bytes_per_call"]), rec["sources_sha256_16"]
    except (KeyError, ValueError):
        return None, "capture summary unreadable"
    if dig != sources_digest():
        return None, "kernel sources changed since the capture"
    return tb, os.path.relpath(TRAFFIC_PROFILE, ROOT)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.samples, self.proc, self.idx = [], None, gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(s[1]) for s in self.samples if len(s) > 2 and s[1].replace(".", "").isdigit()]
        smax = [float(s[2]) for s in self.samples if len(s) > 2 and s[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for k, n in enumerate(names):
                if len(s) > 5 + k and s[5 + k].strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------------------------- oracle
def oracle_triples_sample(fr, t1, t2, jk_pairs):
    """The oracle's (T) pair-matrix work for the given (j,k) pairs (all i, all abc)."""
    from oracle import triples as otr
    ovvv, ovoo, ovov = otr._blocks(fr.B, fr.nocc)
    eo, ev = fr.eps[:fr.nocc], fr.eps[fr.nocc:]
    evs = ev[:, None, None] + ev[None, :, None] + ev[None, None, :]
    tot = 0.0
    for (j, k) in jk_pairs:
        zs, ys = [], []
        for i in range(fr.nocc):
            W = otr.W_block(i, j, k, t2, ovvv, ovoo)
            V = otr.V_block(i, j, k, W, t1, ovov)
            s = np.sqrt(-(eo[i] + eo[j] + eo[k] - evs))
            w, vv = W / s, V / s
            zs.append(4 * w + np.einsum("bca->abc", w) + np.einsum("cab->abc", w))
            ys.append(vv - np.einsum("cba->abc", vv))
        tot += float(np.sum(np.stack(zs) * np.stack(ys)))
    return tot


def cpu_oracle_rate(fr, budget_s=20.0):
    """Time the oracle ((T) work for a few (j,k) pairs of this fragment) and convert to model TFLOP/s."""
    from oracle import ccsd as occ
    t1 = np.zeros((fr.nocc, fr.nvir))
    t2 = occ.mp2_amplitudes(fr.eps, fr.B, fr.nocc)
    pairs, t_used = [], 0.0
    t0 = time.perf_counter()
    j = 0
    while True:
        pairs.append((j % fr.nocc, (j * 7 + 3) % fr.nocc))
        oracle_triples_sample(fr, t1, t2, [pairs[-1]])
        t_used = time.perf_counter() - t0
        j += 1
        if t_used > budget_s * 0.5 or j >= fr.nocc * fr.nocc:
            break
    _, trip = model_flops(fr.nocc, fr.nvir, 0)
    share = len(pairs) / float(fr.nocc * fr.nocc)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": trip * share / t_used / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle (T) pair-matrix work for {len(pairs)} of {fr.nocc**2} (j,k) pairs of the "
                      f"diamond-like fragment ({t_used:.1f} s), scaled by the (T) model flops of those pairs"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed on the host cores on a bounded sample per step."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2407_11258_gb300 import synth
    from oracle import ccsd as occ
    fr = synth.diamond_like()
    t1 = np.zeros((fr.nocc, fr.nvir))
    t2 = occ.mp2_amplitudes(fr.eps, fr.B, fr.nocc)
    _, trip = model_flops(fr.nocc, fr.nvir, 0)
    flops_step = trip / fr.nocc**2
    for w in range(args.warmup):
        oracle_triples_sample(fr, t1, t2, [(w % fr.nocc, (w + 1) % fr.nocc)])
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle_triples_sample(fr, t1, t2, [(k % fr.nocc, (3 * k + 1) % fr.nocc)])
    dt = time.perf_counter() - t0
    val = flops_step * args.steps / dt / 1e12
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = "oracle (T) pair-matrix work for one (j,k) pair of the diamond-like fragment per step"
    print(json.dumps({
        "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


# --------------------------------------------------------------------------------------------- ours
def solve_once(lnocc, fr_dev, opts, stream):
    eps, B, U, o, v, q = fr_dev
    f = lnocc.lnocc_build_ints(o, v, q, eps, B, opts, stream=stream)
    e, it, _ = lnocc.lnocc_ccsd(f, stream=stream)
    ec, em = lnocc.lnocc_fragment_energy(f, U, stream=stream)
    et, etf = lnocc.lnocc_triples(f, U, stream=stream)
    info = f.info()
    f.free()
    return dict(e_ccsd=e, n_iter=it, e_ccsd_frag=ec, e_mp2_frag=em, e_t=et, e_t_frag=etf, e_mp2=info.e_mp2,
                t_gemm_ms=info.t_triples_gemm_ms, t_triples_ms=info.t_triples_ms, launches=info.kernel_launches,
                exec_flops=info.exec_flops)


def batch_measure(lnocc, synth, frag_ids, nfrag, seed, workers, autotune, steps, warmup, stream, sampler=None):
    """Solve fragments `frag_ids` of the uneven batch (nfrag shapes, seed) through lnocc_solve_batch:
    `warmup` untimed batches (the first tunes the tiles when autotune), then `steps` timed ones.
    Returns (seconds per batch, results, input generation seconds)."""
    import torch
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        items = [synth.batch_fragment_device(f, "cuda", nfrag=nfrag, seed=seed) for f in frag_ids]
    stream.synchronize()
    t_gen = time.perf_counter() - t0
    opts = lnocc.default_opts(precision=lnocc.LNOCC_PREC_MIXED, max_iter=200)
    mk = lambda tune: lnocc.default_batch_opts(workers=workers, autotune=tune)  # noqa: E731
    res = None
    for w in range(warmup):
        tune = (1 if w == 0 else 2) if autotune else 0
        _, res = lnocc.lnocc_solve_batch(items, opts, mk(tune), stream=stream, allow_noconv=True)
    torch.cuda.synchronize()
    times = []
    with (sampler if sampler is not None else contextlib.nullcontext()):
        for _ in range(steps):
            t1 = time.perf_counter()
            _, res = lnocc.lnocc_solve_batch(items, opts, mk(2 if autotune else 0), stream=stream, allow_noconv=True)
            times.append(time.perf_counter() - t1)
    del items
    return float(np.mean(times)), res, t_gen


def run_batch(args):
    """Uneven-fragment batch through lnocc_solve_batch; one step = the whole batch. With N ranks the one
    fragment list is split by LPT on the runtime's own cost model (shard.assign): each rank solves its
    share, the energies are gathered and summed in fragment order (strong scaling, no collective in the
    data path)."""
    import torch
    from paper_2407_11258_gb300 import build, lnocc, shard, synth
    world, rank, local = dist_setup()
    build.build()
    lnocc.load()
    stream = torch.cuda.Stream()
    seed = 3000
    shapes = synth.batch_shapes(args.nfrag, seed)
    mine = shard.assign([(o, v, q, synth.batch_gap(f, args.nfrag, seed)) for f, (o, v, q, _) in enumerate(shapes)],
                        world)[rank]
    barrier(world)
    sampler = ClockSampler(local)
    sec, res, t_gen = batch_measure(lnocc, synth, mine, args.nfrag, seed, args.workers, args.autotune, args.steps,
                                    args.warmup, stream, sampler)
    if args.autotune and args.save_tune:
        lnocc.lnocc_autotune_save(args.save_tune)
    barrier(world)
    sec = max_over_ranks(world, sec)
    local_e = {f: (r.e_ccsd + r.e_t, r.model_flops, r.status, r.n_iter) for f, r in zip(mine, res)}
    allE = shard.gather_energies(local_e, world)
    if rank != 0:
        return
    flops = sum(x[1] for x in allE.values())
    peak_burst, peak_sust, hbm, peak_src = read_peaks()
    achieved = flops / sec / 1e12
    n_ok = sum(x[2] == lnocc.LNOCC_OK for x in allE.values())
    busy = sum(r.t_end_ms - r.t_start_ms for r in res) / 1e3
    print(json.dumps({
        "metric": METRIC, "value": achieved, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "bf16x3/fp32 (fp64 update, DIIS, energies)", "data": "synthetic",
        "config": {"workload": f"uneven batch of {args.nfrag} fragments: nocc U{{8..24}}, nvir U{{120..360}}, "
                               f"naux=4*nvir, half small-gap (seed {seed}); LPT split over {world} rank(s)",
                   "l2": "inputs (88 GB for 128 fragments) far larger than L2; no flush",
                   "workers": args.workers, "autotune": args.autotune},
        "solves_per_s": len(allE) / sec, "converged": n_ok, "n_frag": len(allE),
        "sum_e_ccsd_plus_t_ordered": shard.ordered_sum({f: x[0] for f, x in allE.items()}),
        "mean_ccsd_iterations": float(np.mean([x[3] for x in allE.values()])),
        "not_converged": [{"frag": f, "status": x[2], "n_iter": x[3], "shape": list(shapes[f])}
                          for f, x in sorted(allE.items()) if x[2] != lnocc.LNOCC_OK],
        "pipeline_occupancy_rank0": busy / sec,
        "input_generation_s_rank0": t_gen,
        "e2e": None, "e2e_note": "not measured for the batch workload (88 GB of inputs)",
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_burst / 3.0, "unit": "TFLOP/s",
                     "frac": achieved / (peak_burst / 3.0), "traffic": None,
                     "kernel": "whole batch (model flops / wall time)",
                     "note": f"peak = {peak_src} bf16 burst {peak_burst} / 3 (BF16x3)"},
        "autotune_stats": lnocc.lnocc_autotune_stats(),
        "clocks": sampler.summary(),
    }), flush=True)


def triples_measure(lnocc, synth, rank=0, sampler=None):
    """(T)-dominated fragment nocc=32, nvir=480, naux=1600 (B drawn on the device): one mixed solve with
    (T) timed by the library's CUDA events; then the scaled fragment nocc=12, nvir=96, naux=320 against
    the stored oracle energies (tests/golden/make_golden.py wrote them from the oracle; the full-size
    oracle (T) would take days)."""
    import torch
    o, v, q = 32, 480, 1600
    item = synth.fragment_device(o, v, q, False, 4000 + rank, "cuda", frag=(0,))
    _, _, _, eps, B, U = item
    opts = lnocc.default_opts(precision=lnocc.LNOCC_PREC_MIXED)
    t0 = time.perf_counter()
    f = lnocc.lnocc_build_ints(o, v, q, eps, B, opts)
    del item, B
    t1 = time.perf_counter()
    e, it, _ = lnocc.lnocc_ccsd(f, allow_noconv=True)
    t2 = time.perf_counter()
    with (sampler if sampler is not None else contextlib.nullcontext()):
        et, etf = lnocc.lnocc_triples(f, U)
    t3 = time.perf_counter()
    info = f.info()
    f.free()
    torch.cuda.empty_cache()
    _, trip = model_flops(o, v, 0)
    alg = triples_algorithmic_flops(o, v)
    ref = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_small.json")))["triples_scaled"]
    frs = synth.triples_large(scaled=True)
    eps_s, B_s, U_s = (torch.tensor(x, device="cuda") for x in (frs.eps, frs.B, frs.U_frag))
    fs = lnocc.lnocc_build_ints(frs.nocc, frs.nvir, frs.naux, eps_s, B_s, opts)
    es, _, _ = lnocc.lnocc_ccsd(fs, allow_noconv=True)
    ets, etfs = lnocc.lnocc_triples(fs, U_s)
    fs.free()
    return {
        "workload": "(T)-dominated fragment nocc=32 nvir=480 naux=1600, 1 LMO",
        "triples_ms": info.t_triples_ms, "contraction_ms": info.t_triples_gemm_ms,
        "model_tflops": trip / (info.t_triples_ms * 1e-3) / 1e12,
        "executed_contraction_tflops": alg / (info.t_triples_gemm_ms * 1e-3) / 1e12,
        "energies": {"e_ccsd": e, "e_t": et, "e_t_frag": etf}, "ccsd_iterations": it,
        "t_build_s": t1 - t0, "t_ccsd_s": t2 - t1, "t_triples_wall_s": t3 - t2, "device_gb": info.device_bytes / 1e9,
        "scaled_size": {"workload": "nocc=12 nvir=96 naux=320", "abs_err_vs_oracle": {
            "e_ccsd": abs(es - ref["e_ccsd"]), "e_t": abs(ets - ref["e_t"]), "e_t_frag": abs(etfs - ref["e_t_frag"])}},
    }


def run_triples(args):
    """The (T)-dominated fragment as its own bench line."""
    from paper_2407_11258_gb300 import build, lnocc, synth
    world, rank, local = dist_setup()
    build.build()
    lnocc.load()
    sampler = ClockSampler(local)
    r = triples_measure(lnocc, synth, rank, sampler)
    if rank != 0:
        return
    peak_burst, peak_sust, hbm, peak_src = read_peaks()
    achieved = r["executed_contraction_tflops"]
    print(json.dumps({
        "metric": METRIC, "value": r["model_tflops"], "unit": "TFLOP/s ((T) model flops)",
        "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": r["triples_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3/fp32 (fp64 denominators and energy sum)",
        "data": "synthetic", "config": {"workload": r["workload"]}, "triples": r,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_burst / 3.0, "unit": "TFLOP/s",
                     "frac": achieved / (peak_burst / 3.0), "traffic": None,
                     "kernel": "k_gemm_tc ((T) W contractions)", "raw_bf16_tflops": 3.0 * achieved,
                     "note": f"useful 2o^3v^4+2o^4v^3 / contraction event time; peak = {peak_src} bf16 burst / 3"},
        "clocks": sampler.summary(),
    }), flush=True)


def mlp_measure(lnocc, synth, ntrain, nheld, nheld_fp64, train_steps, batch, prec):
    """Learned T2 guess: generate training solves on the GPU, train the MLP with the library's kernels,
    then solve held-out fragments from the MP2 guess and from the learned guess (and nheld_fp64 of them
    again on the FP64 path, where converged energies compare at 1e-8 Eh)."""
    import torch
    dev = "cuda"
    per_frag = 4096
    t0 = time.perf_counter()
    Xs, dts, it_train = [], [], []
    for k in range(ntrain):
        o, v, q, eps, B, U = synth.mlp_fragment_device(k, dev)
        f = lnocc.lnocc_build_ints(o, v, q, eps, B, lnocc.default_opts(precision=prec))
        _, it, _ = lnocc.lnocc_ccsd(f, allow_noconv=True)
        it_train.append(it)
        gen = torch.Generator(device=dev)
        gen.manual_seed(100 + k)
        idx = torch.randint(0, o * o * v * v, (per_frag,), generator=gen, device=dev, dtype=torch.int64)
        X = torch.empty(per_frag, 8, dtype=torch.float32, device=dev)
        dt = torch.empty(per_frag, dtype=torch.float32, device=dev)
        lnocc.lnocc_mlp_samples(f, idx, X, dt)
        Xs.append(X)
        dts.append(dt)
        f.free()
        del B
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    X, dt = torch.cat(Xs), torch.cat(dts)
    m = lnocc.Mlp(synth.mlp_init(5100))
    m.fit_norm(X, dt)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    t0 = time.perf_counter()
    losses = []
    for step in range(train_steps):
        sel = torch.randint(0, X.shape[0], (batch,), generator=gen, device=dev)
        lr = 3e-3 if step < 0.7 * train_steps else 1e-3
        losses.append(m.train_step(X[sel].contiguous(), dt[sel].contiguous(), lr))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    it0, it1, t_mp2, t_mlp, de, fallbacks, noconv = [], [], [], [], [], 0, []
    for k in range(2000, 2000 + nheld):
        o, v, q, eps, B, U = synth.mlp_fragment_device(k, dev)
        f = lnocc.lnocc_build_ints(o, v, q, eps, B, lnocc.default_opts(precision=prec))
        lnocc.lnocc_frag_set_mlp(f, m)
        torch.cuda.synchronize()
        a = time.perf_counter()
        e0, n0, s0 = lnocc.lnocc_ccsd(f, allow_noconv=True)
        b = time.perf_counter()
        e1, n1, s1 = lnocc.lnocc_ccsd(f, guess_mode=lnocc.LNOCC_GUESS_MLP, allow_noconv=True)
        c = time.perf_counter()
        it0.append(n0)
        it1.append(n1)
        t_mp2.append(b - a)
        t_mlp.append(c - b)
        # energies compare where both solves converged; a solve stopped at the mixed noise floor
        # (ENOCONV, energy spread above 1e-7 Eh) is counted apart
        if s0 == lnocc.LNOCC_OK and s1 == lnocc.LNOCC_OK:
            de.append(abs(e1 - e0))
        else:
            noconv.append((k, int(s0), int(s1), abs(e1 - e0)))
        f.free()
    # the same comparison on the FP64 path, where converged energies can be compared at 1e-8 Eh
    it0_64, it1_64, de_64 = [], [], []
    for k in range(2000, 2000 + nheld_fp64):
        o, v, q, eps, B, U = synth.mlp_fragment_device(k, dev)
        f = lnocc.lnocc_build_ints(o, v, q, eps, B, lnocc.default_opts(precision=lnocc.LNOCC_PREC_FP64))
        lnocc.lnocc_frag_set_mlp(f, m)
        e0, n0, _ = lnocc.lnocc_ccsd(f, allow_noconv=True)
        e1, n1, _ = lnocc.lnocc_ccsd(f, guess_mode=lnocc.LNOCC_GUESS_MLP, allow_noconv=True)
        it0_64.append(n0)
        it1_64.append(n1)
        de_64.append(abs(e1 - e0))
        f.free()
    m.free()
    return {
        "workload": f"learned T2 guess: {ntrain} training solves, {nheld} held-out fragments, nocc U{{8..16}}, "
                    f"nvir U{{96..240}}, naux=4*nvir, half small-gap",
        "precision": "mixed" if prec else "fp64", "samples_per_fragment": per_frag, "train_steps": train_steps,
        "batch": batch, "n_held": nheld,
        "mean_iterations_mp2_guess": float(np.mean(it0)), "mean_iterations_mlp_guess": float(np.mean(it1)),
        "mean_ccsd_s_mp2_guess": float(np.mean(t_mp2)), "mean_ccsd_s_mlp_guess": float(np.mean(t_mlp)),
        "held_out_solves_per_s_mlp_guess": nheld / sum(t_mlp),
        "max_abs_dE_mlp_vs_mp2_guess": float(np.max(de)) if de else None,
        "n_both_converged": len(de),
        "noise_floor_stops": {"count": len(noconv),
                              "max_abs_dE": float(max(x[3] for x in noconv)) if noconv else None,
                              "note": "fragments where either solve stopped at the mixed noise floor (ENOCONV: "
                                      "energy spread > 1e-7 Eh; opts.n_refine would refine them in FP64)"},
        "fp64_path": {"n_frag": nheld_fp64,
                      "mean_iterations_mp2_guess": float(np.mean(it0_64)) if it0_64 else None,
                      "mean_iterations_mlp_guess": float(np.mean(it1_64)) if it1_64 else None,
                      "max_abs_dE_mlp_vs_mp2_guess": float(np.max(de_64)) if de_64 else None},
        "train_loss_first": float(np.mean(losses[:10])), "train_loss_last": float(np.mean(losses[-50:])),
        "t_training_data_s": t_data, "t_training_s": t_train,
        "mean_iterations_training_solves": float(np.mean(it_train)),
    }


def run_mlp(args):
    """The learned-guess workload as its own bench line."""
    from paper_2407_11258_gb300 import build, lnocc, synth
    world, rank, local = dist_setup()
    build.build()
    lnocc.load()
    prec = lnocc.LNOCC_PREC_MIXED if args.mlp_precision == "mixed" else lnocc.LNOCC_PREC_FP64
    r = mlp_measure(lnocc, synth, args.ntrain, args.nheld, args.nheld_fp64, args.train_steps, args.batch, prec)
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": r["held_out_solves_per_s_mlp_guess"],
        "unit": "CCSD solves/s (held-out, learned guess)", "n_gpus": world, "steps": args.nheld, "warmup": 0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3/fp32" if prec else "f64", "data": "synthetic",
        "config": {"workload": r["workload"]}, "mlp": r}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--workload", default="diamond", choices=["diamond", "batch", "mlp", "triples", "case"])
    ap.add_argument("--extras", default="all", choices=["all", "none"],
                    help="diamond workload: also measure the reduced batch, the (T)-dominated fragment and the "
                         "learned guess (bounded; outside the timed region)")
    ap.add_argument("--extra-batch", type=int, default=16, help="fragments of the reduced batch extra")
    ap.add_argument("--nocc", type=int, default=16, help="case workload: occupied orbitals")
    ap.add_argument("--nvir", type=int, default=120, help="case workload: virtual orbitals")
    ap.add_argument("--naux", type=int, default=480, help="case workload: auxiliary functions")
    ap.add_argument("--iters", type=int, default=4, help="case workload: CCSD iteration cap")
    ap.add_argument("--fp64", action="store_true", help="case workload: plain FP64 path")
    ap.add_argument("--mlp-guess", action="store_true", help="case workload: also run the learned-guess kernel once")
    ap.add_argument("--tchunk", type=int, default=0, help="case workload: (T) W chunk bound in MB (0: library default)")
    ap.add_argument("--tkernel", type=int, default=0,
                    help="case workload: (T) contraction launches (0 auto, 1 one per term, 2 grouped)")
    ap.add_argument("--repeat", type=int, default=1, help="case workload: lnocc_triples calls (the last one is printed)")
    ap.add_argument("--ntrain", type=int, default=2000, help="mlp workload: training solves")
    ap.add_argument("--nheld", type=int, default=256, help="mlp workload: held-out fragments")
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--mlp-precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--nheld-fp64", type=int, default=16, help="mlp workload: held-out fragments also run in FP64")
    ap.add_argument("--nfrag", type=int, default=128, help="batch workload: fragments per batch")
    ap.add_argument("--workers", type=int, default=0, help="batch workload: concurrent pipelines (0: library default)")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1], help="batch workload: tile autotuning")
    ap.add_argument("--tune", action="store_true", help="diamond workload: tile autotuning during warm-up")
    ap.add_argument("--save-tune", default=None, help="write the tile table to this file after tuning")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "mlp":
        return run_mlp(args)
    if args.workload == "triples":
        return run_triples(args)
    if args.workload == "case":
        return run_case(args)

    import torch
    from paper_2407_11258_gb300 import build, lnocc, synth
    world, rank, local = dist_setup()
    build.build()
    lnocc.load()
    stream = torch.cuda.Stream()
    # independent fragments per rank (weak scaling): rank r solves the diamond-like fragment with seed 2000+r
    fr = synth.diamond_like(seed=2000 + rank)
    o, v, q = fr.nocc, fr.nvir, fr.naux
    eps_h = torch.tensor(fr.eps).pin_memory()
    B_h = torch.tensor(fr.B).pin_memory()
    U_h = torch.tensor(fr.U_frag).pin_memory()
    with torch.cuda.stream(stream):
        eps_d, B_d, U_d = eps_h.cuda(non_blocking=True), B_h.cuda(non_blocking=True), U_h.cuda(non_blocking=True)
    stream.synchronize()
    opts = lnocc.default_opts(precision=lnocc.LNOCC_PREC_MIXED)
    fr_dev = (eps_d, B_d, U_d, o, v, q)
    for w in range(args.warmup):
        if args.tune:  # the first warm-up solve times the tile candidates; later solves use the table
            lnocc.lnocc_autotune(2 if w == 0 else 1)
        res = solve_once(lnocc, fr_dev, opts, stream)
    if args.tune and args.save_tune:
        lnocc.lnocc_autotune_save(args.save_tune)
    # ---- device-resident timed region
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    with sampler:
        ev0.record(stream)
        runs = [solve_once(lnocc, fr_dev, opts, stream) for _ in range(args.steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(world, ms)
    n_iter = runs[-1]["n_iter"]
    ccsd_f, trip_f = model_flops(o, v, n_iter)
    flops_solve = ccsd_f + trip_f
    tflops = world * flops_solve / (ms * 1e-3) / 1e12
    launches = runs[-1]["launches"] - res["launches"]  # library-wide launch counter across the timed steps
    # ---- end to end: pinned host inputs copied in, energies read back, every step
    e2e_ms = None
    h2d = (eps_h.numel() + B_h.numel() + U_h.numel()) * 8
    t0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            eps_x = eps_h.cuda(non_blocking=True)
            B_x = B_h.cuda(non_blocking=True)
            U_x = U_h.cuda(non_blocking=True)
        solve_once(lnocc, (eps_x, B_x, U_x, o, v, q), opts, stream)
        del eps_x, B_x, U_x
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(world, (time.perf_counter() - t0) / args.steps * 1e3)
    if rank != 0:
        return
    # ---- roofline of the dominant kernel: the (T) tensor-core contractions (event-timed per chunk)
    peak_burst, peak_sust, hbm, peak_src = read_peaks()
    gemm_ms = float(np.mean([r["t_gemm_ms"] for r in runs]))
    alg = triples_algorithmic_flops(o, v)
    achieved = alg / (gemm_ms * 1e-3) / 1e12
    peak = peak_burst / 3.0  # BF16x3: three bf16 products per useful product
    traffic, traffic_src = recorded_traffic()
    out = {
        "metric": METRIC, "value": tflops, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3/fp32 (fp64 update, DIIS, energies)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "inputs (0.5 GB B tensor) larger than L2; no flush",
                   "ccsd_iterations": n_iter, "tile_autotune": bool(args.tune)},
        "solves_per_s": world * 1e3 / ms,
        "executed_contraction_tflops": world * runs[-1]["exec_flops"] / (ms * 1e-3) / 1e12,
        "executed_note": "contraction flops the kernels issue per solve (the library's count: each BF16x3 product "
                         "once; (T) on sorted virtual triples, the ladder on packed +/- pairs) over the same time; "
                         "`value` counts the paper's work model 2o^2v^4+16o^3v^3+2o^4v^2 per iteration + "
                         "6o^3v^4+6o^4v^3",
        "energies": {k: runs[-1][k] for k in ("e_mp2", "e_ccsd", "e_ccsd_frag", "e_mp2_frag", "e_t", "e_t_frag")},
        "e2e": {"value": world * flops_solve / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 6 * 8},
        "gpu_launches": launches,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                     "traffic_unit": "DRAM bytes read + written by the k_gemm_tc launches of one lnocc_triples call",
                     "kernel": "k_gemm_tc ((T) W contractions)",
                     "note": f"useful (T) contraction flops 2o^3v^4+2o^4v^3 per call / event time of those launches; "
                             f"peak = {peak_src} bf16 burst {peak_burst} / 3 (BF16x3)",
                     "triples_ms": float(np.mean([r['t_triples_ms'] for r in runs])), "contraction_ms": gemm_ms,
                     "raw_bf16_tflops": 3.0 * achieved},
        "clocks": sampler.summary(),
    }
    ref_path = os.path.join(ROOT, "tests", "golden", "oracle_diamond.json")
    if os.path.exists(ref_path) and rank == 0:
        ref = json.load(open(ref_path))["diamond_like"]
        out["abs_err_vs_oracle"] = {k: abs(runs[-1][k] - ref[k]) for k in out["energies"] if k in ref}
    if not args.no_fp64:
        opts64 = lnocc.default_opts(precision=lnocc.LNOCC_PREC_FP64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r64 = solve_once(lnocc, fr_dev, opts64, stream)
        t64 = time.perf_counter() - t0
        ccsd64, _ = model_flops(o, v, r64["n_iter"])
        out["fp64_gpu"] = {"ms_per_solve": t64 * 1e3, "value": (ccsd64 + trip_f) / t64 / 1e12, "unit": "TFLOP/s",
                           "speedup_mixed_vs_fp64": t64 * 1e3 / ms, "n_iter": r64["n_iter"],
                           "abs_diff_vs_mixed": {k: abs(r64[k] - runs[-1][k]) for k in out["energies"]}}
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_oracle_rate(fr)
    if args.extras == "all":
        out["extras"] = run_extras(lnocc, synth, args, stream)
    print(json.dumps(out), flush=True)


def run_extras(lnocc, synth, args, stream):
    """The other workloads of the metric, bounded so that the default run stays within minutes; each is
    measured outside the timed region above (after it) and reported under its own key."""
    import torch
    from paper_2407_11258_gb300 import shard
    ex = {}
    torch.cuda.empty_cache()
    # uneven batch: the first extra_batch fragments of the 128-fragment list (half small-gap), one timed batch
    nb = args.extra_batch
    t0 = time.perf_counter()
    sec, res, t_gen = batch_measure(lnocc, synth, list(range(nb)), 128, 3000, 0, 1, 1, 1, stream)
    flops = sum(r.model_flops for r in res)
    ex["batch_reduced"] = {
        "workload": f"first {nb} of the 128 uneven batch fragments (nocc U{{8..24}}, nvir U{{120..360}}, naux=4*nvir, "
                    f"odd index small-gap), lnocc_solve_batch, 1 warm-up + 1 timed batch",
        "seconds": sec, "solves_per_s": nb / sec, "model_tflops": flops / sec / 1e12,
        "converged": sum(r.status == lnocc.LNOCC_OK for r in res), "n_frag": nb,
        "mean_ccsd_iterations": float(np.mean([r.n_iter for r in res])),
        "max_ccsd_iterations": int(max(r.n_iter for r in res)),
        "sum_e_ccsd_plus_t_ordered": shard.ordered_sum({k: r.e_ccsd + r.e_t for k, r in enumerate(res)}),
        "wall_s": time.perf_counter() - t0}
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    ex["triples_large"] = triples_measure(lnocc, synth)
    ex["triples_large"]["wall_s"] = time.perf_counter() - t0
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    ex["learned_guess"] = mlp_measure(lnocc, synth, args.ntrain, args.nheld, args.nheld_fp64, args.train_steps,
                                      args.batch, lnocc.LNOCC_PREC_MIXED)
    ex["learned_guess"]["wall_s"] = time.perf_counter() - t0
    return ex


def run_case(args):
    """One fragment solve through the C-ABI with the library's own timings printed (for profiling with
    external tools such as ncu): integrals, up to --iters CCSD iterations (mixed unless --fp64), the
    fragment energies, optionally one learned-guess inference, then the (T) energy."""
    import torch
    from paper_2407_11258_gb300 import build, lnocc, synth
    build.build()
    lnocc.load()
    o, v, q = args.nocc, args.nvir, args.naux
    fr = synth.make_fragment(o, v, q, 2024, decay=20.0, frag=(0, 1) if o > 1 else (0,))
    eps, B, U = (torch.tensor(x, device="cuda") for x in (fr.eps, fr.B, fr.U_frag))
    prec = lnocc.LNOCC_PREC_FP64 if args.fp64 else lnocc.LNOCC_PREC_MIXED
    f = lnocc.lnocc_build_ints(o, v, q, eps, B, lnocc.default_opts(precision=prec, max_iter=args.iters,
                                                                     triples_chunk_mb=args.tchunk,
                                                                     triples_kernel=args.tkernel))
    t0 = time.perf_counter()
    e, it, _ = lnocc.lnocc_ccsd(f, allow_noconv=True)
    t1 = time.perf_counter()
    ec, em = lnocc.lnocc_fragment_energy(f, U)
    out = f"ccsd {it} iterations {1e3 * (t1 - t0):.1f} ms E={e:.12f} E_frag={ec:.12f}"
    if args.mlp_guess:
        m = lnocc.Mlp(synth.mlp_init())
        t2g = torch.empty(o, o, v, v, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        tg = time.perf_counter()
        lnocc.lnocc_mlp_guess(f, m, t2g)
        torch.cuda.synchronize()
        out += f"; learned guess {1e3 * (time.perf_counter() - tg):.2f} ms"
        m.free()
    for _ in range(max(1, args.repeat)):
        et, etf = lnocc.lnocc_triples(f, U)
    inf = f.info()
    out += (f"; (T) chunk {args.tchunk or 768} MB: device {inf.t_triples_ms:.1f} ms (contractions "
            f"{inf.t_triples_gemm_ms:.1f} ms)"
            f" E_T={et:.12f} E_T_frag={etf:.12f}")
    f.free()
    print(out, flush=True)


if __name__ == "__main__":
    main()
