"""Benchmark: encrypted semi-parallel GWAS throughput (SNPs/s) on GB300.

One step = one whole encrypted job of the paper's shape (245 samples,
intercept + 4 covariates, 10643 SNPs; CKKS N = 2^16, 24 q-limbs, 8 special
primes, dnum = 3, kappa = 1): encrypt the inputs (X, (X^T X)^-1, y and all
42 SNP batches), the encrypted covariate fit (Alg. 9-10, z, z'), every SNP
batch (Alg. 11 loop) and the decryption of all numerators / denominators.
Keys are generated once, outside the timed region.

  value      inputs already resident in HBM (torch tensors), CUDA events on the
             library's stream, L2 flushed (256 MiB write) between steps
  e2e        the same job through the C ABI with pinned host inputs: the
             host->device copies and the result read-back are inside the timing
  phases_ms  the paper's phases (context generation, encryption, computations,
             decryption; tables speed-mem-seal / speed-mem-heaan) from one job
             run through the split boundary calls, checked equal to the fused job
  roofline   the dominant kernel class from the library's event timers, on one
             extra instrumented step; per-class achieved GB/s beside it
  mccp       the paper's own M-CCP layout (Alg. 11) timed the same way, with
             Dup(M_j) in HBM and in the pinned host tier
  micro      kernel microbench: 3072 limb transforms, 512 level-24 rotations
             with rescale as batched sets (key-switch roofline), hoisted sums
  cpu_baseline  the CPU oracle on a bounded sample (one key switch at every
             level the job switches at, on all host cores and on one thread;
             one tensor and one encryption at the batch level) extrapolated to
             the job with its key-switch histogram; beside it the plaintext
             FP64 GWAS of the same inputs, against which the timed job's
             decrypted statistics are checked, and the paper's accuracy report
             against the exact semi-parallel method

Multi-GPU (torchrun): every rank runs its own independent job (weak scaling),
no collective on the data path; value = SNPs of all ranks / max step time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted-GWAS SNPs/s (245 samples, N=2^16); key-switch/s vs HBM roofline"
WORKLOAD = dict(name="paper-n245", logN=16, L=24, q0_bits=60, scale_bits=45, K=8, sp_bits=60,
                dnum=3, n=245, d=5, k=10643, seed=1002, kappa=1)
# the paper's own ring and its most accurate fit (kappa = 3): N = 2^17, 40 limbs
WORKLOAD_K3 = dict(name="paper-n245-kappa3", logN=17, L=40, q0_bits=60, scale_bits=45, K=12,
                   sp_bits=60, dnum=3, n=245, d=5, k=10643, seed=1006, kappa=3)
BENCH_WORKLOADS = {"paper-n245": WORKLOAD, "paper-n245-kappa3": WORKLOAD_K3}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except Exception:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# GB300: 152 SMs of four sub-partitions, each with one fmaheavy pipe (the
# only pipe that executes integer multiply-adds).  The butterfly (estimated
# Shoup product + lazy corrections) occupies that pipe for
# FMAHEAVY_CYCLES_PER_WARP_BFLY cycles per 32 butterflies (one per lane):
# measured by ncu on the register-only probe (sm__pipe_fmaheavy_cycles_active
# 95.05% of 38.3 M cycles per sub-partition for 1.05 M warp-butterflies each).
# The probe's 23.8 warp instructions per warp-butterfly would allow more, so
# the multiply-add pipe, not issue, bounds the transform.
NUM_SMS = 152
FMAHEAVY_CYCLES_PER_WARP_BFLY = 34.7
# ncu, 3072 rows of 2^16 in shape 4 (profiles/ntt_pass_ntt-ks-micro.md): DRAM
# read + write of pass A 1.611 + 1.555 GB, pass B 1.858 + 1.561 GB
NTT_DRAM_BYTES_PER_LIMB = round((1.611e9 + 1.555e9 + 1.858e9 + 1.561e9) / 3072)


def alu_peak_gbfly(sm_mhz):
    """multiply-add-pipe bound of the butterfly rate (G/s) at the given SM clock."""
    return NUM_SMS * 4 * sm_mhz * 1e6 * 32.0 / FMAHEAVY_CYCLES_PER_WARP_BFLY / 1e9


def client_preprocess(X):
    """Client-side plaintext pre-processing of the paper (section 'Hessian
    Matrix Approximation'): (X^T X)^-1, computed before encryption."""
    return np.linalg.inv(X.T @ X)


def _event_maker(stream):
    import torch

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e
    return ev


def class_rates(prof):
    """per kernel class: event time (ms), algorithmic bytes / time (GB/s),
    launch groups"""
    return {k: {"ms": round(v[0], 3),
                "gbs": round(v[1] / (v[0] / 1e3) / 1e9, 1) if v[0] > 0 else None,
                "launch_groups": int(v[2])} for k, v in prof.items()}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_1902_04303_gb300 import build as pkg_build
    from paper_1902_04303_gb300 import gwhe
    from paper_1902_04303_gb300.datagen import make_gwas

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    pkg_build.build()
    W = BENCH_WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    ev = _event_maker(stream)
    # --shard-job: the ranks share one job (same keys and inputs), rank 0 fits
    # and broadcasts the batch-invariant state, each evaluates its batch range
    shard = bool(args.shard_job)
    # context generation (the paper's phase): tables, then every key the job needs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = gwhe.Context(W["logN"], W["L"], W["q0_bits"], W["scale_bits"], W["K"], W["sp_bits"],
                       W["dnum"], seed=W["seed"] + (0 if shard else 7919 * rank),
                       stream=stream.cuda_stream)
    probe = gwhe.Job(ctx, W["n"], W["d"], W["k"], layout=args.layout)
    steps_rot, layout_used = probe.rotation_steps(), "factored" if probe.factored else "mccp"
    probe.close()
    ctx.keygen(rot_steps=steps_rot, conj=True)
    torch.cuda.synchronize()
    t_ctxgen = time.perf_counter() - t0
    # the fastest compiled shapes of the transform on this GPU, for large
    # launches and for those of a few waves or less
    tuned = ctx.autotune()
    tuned_small = ctx.autotune(rows=32)
    if args.ntt_shape >= 0:
        # a fixed shape (profiler captures, whose serialised launches would
        # mislead the autotuner)
        ctx.set_ntt_variant(args.ntt_shape)
        tuned = (args.ntt_shape, tuned[1])
        tuned_small = (args.ntt_shape, tuned_small[1])
    data = make_gwas(W["n"], W["d"], W["k"], seed=W["seed"] + (0 if shard else rank))
    A = client_preprocess(data.X)
    dev = {nm: torch.from_numpy(np.ascontiguousarray(v)).cuda()
           for nm, v in (("X", data.X), ("A", A), ("y", data.y), ("S", data.S))}
    host = {nm: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
            for nm, v in (("X", data.X), ("A", A), ("y", data.y), ("S", data.S))}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(src, layout=args.layout, host_state=args.host_state):
        if shard:
            from paper_1902_04303_gb300.sharding import run_sharded_job
            job = gwhe.Job(ctx, W["n"], W["d"], W["k"], layout=layout)
            num, den, _ = run_sharded_job(ctx, job, src["X"], src["A"], src["y"], src["S"],
                                          W["kappa"], rank, world, device="cuda")
            job.close()
            return num, den
        job = gwhe.Job(ctx, W["n"], W["d"], W["k"], layout=layout)
        if host_state:
            job.set_host_state(host_state)  # Dup(M_j) in pinned host memory
        job.encrypt_inputs(src["X"], src["A"], src["y"])
        if job.factored:
            # SNP batches encrypted first: the fit computes their S' beside
            # the covariate phase
            job.encrypt_snps(src["S"])
            job.fit(W["kappa"])
            job.snp_stats(None)
        else:
            job.fit(W["kappa"])
            job.snp_stats(src["S"])
        num, den = job.decrypt_results()
        job.close()
        return num, den

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def timed(src, K, **kw):
        ms = []
        barrier()
        for _ in range(K):
            flush.zero_()
            # NVTX range around each timed job: profilers can select exactly
            # these launches (ncu --nvtx --nvtx-include "gwas_job/")
            torch.cuda.nvtx.range_push("gwas_job")
            e0 = ev()
            out = step(src, **kw)
            e1 = ev()
            torch.cuda.nvtx.range_pop()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        barrier()
        return ms, out

    for _ in range(args.warmup):
        step(dev)
    ks0, l0 = ctx.ks_histogram().copy(), ctx.launches()
    with Clocks(local) as clk:
        ms, (num, den) = timed(dev, args.steps)
    ks_hist = (ctx.ks_histogram() - ks0) // args.steps
    launches = ctx.launches() - l0
    ks_all = int(ks_hist.sum())  # key switches per step over all ranks
    if world > 1:
        t = torch.tensor([float(ks_all)], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        ks_all = int(t.item())
    step_ms = float(np.mean(ms))
    if world > 1:
        t = torch.tensor([step_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms = float(t.item())
    # the context's pinned staging buffers for host genotypes are allocated by
    # its first host-input job (once, like the keys): one untimed step
    step(host)
    ms_e2e, _ = timed(host, max(1, args.steps))
    e2e_ms = float(np.mean(ms_e2e))
    if world > 1:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())

    # the paper's phases through the split boundary calls (encryption of the
    # inputs and of every SNP batch, then the computations on them, then the
    # decryption); the job must give the fused job's statistics bit for bit
    def split_step():
        job = gwhe.Job(ctx, W["n"], W["d"], W["k"], layout=args.layout)
        if args.host_state:
            job.set_host_state(args.host_state)
        flush.zero_()
        e = [ev()]
        job.encrypt_covariates(dev["X"], dev["A"])
        job.encrypt_phenotype(dev["y"])
        job.encrypt_snps(dev["S"])
        e.append(ev())
        job.fit(W["kappa"])
        job.snp_stats(None)
        e.append(ev())
        sn, sd = job.decrypt_results()
        e.append(ev())
        job.close()
        e[-1].synchronize()
        return [e[i].elapsed_time(e[i + 1]) for i in range(3)], sn, sd

    split_step()
    ph, sn, sd = split_step()
    phases = {"context_generation_ms": round(t_ctxgen * 1e3, 1),
              "encryption_ms": round(ph[0], 3), "computations_ms": round(ph[1], 3),
              "decryption_ms": round(ph[2], 3),
              "split_equals_fused": bool(np.array_equal(sn, num, equal_nan=True) and
                                         np.array_equal(sd, den, equal_nan=True)),
              "computations_snps_per_s": round(W["k"] / (ph[1] / 1e3), 1)}

    # one instrumented step for the per-kernel roofline
    ctx.prof_enable(True)
    step(dev)
    prof = ctx.prof_read()
    ctx.prof_enable(False)

    # the paper's own layout (Alg. 11, M in CCP form), on the device and with
    # Dup(M_j) in the pinned host tier
    mccp = None
    if layout_used == "factored" and not args.no_mccp:
        mccp = {}
        for nm, hs in (("hbm", 0), ("host_tier_32", 32)):
            step(dev, layout="mccp", host_state=hs)
            mm, _ = timed(dev, max(1, min(3, args.steps)), layout="mccp", host_state=hs)
            t = float(np.mean(mm))
            mccp[nm] = {"ms_per_job": round(t, 3), "snps_per_s": round(W["k"] / (t / 1e3), 1)}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    snps = W["k"] * (1 if shard else world)
    value = snps / (step_ms / 1e3)
    ks_per_job = int(ks_hist.sum())
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    dom = max(prof, key=lambda k: prof[k][0])
    ms_d, by_d, cnt_d = prof[dom]
    achieved = by_d / (ms_d / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel_class": dom, "achieved": round(achieved, 1), "peak": hbm,
            "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": None,
            "peak_source": "measured" if "hbm_gbs" in pk else "fallback",
            "launch_groups": cnt_d, "ms_per_step": round(ms_d, 3),
            "share_of_step": round(ms_d / sum(v[0] for v in prof.values()), 3),
            "classes": class_rates(prof)}
    clk_mhz = clk.summary().get("sm_max_mhz") or 2070.0
    if dom == "ntt":
        # the NTT is bound by 64-bit modular arithmetic: report it against the
        # butterfly issue ceiling (unit counts x clock / instructions per
        # butterfly), with the register-only probe and the HBM view beside it
        bfly = by_d / 16.0 * (W["logN"] / 2.0)  # 16 B and N/2 log2 N butterflies per limb row
        ach_b = bfly / (ms_d / 1e3) / 1e9
        probe, _ = ctx.probe_butterflies()
        peak_b = alu_peak_gbfly(clk_mhz)
        roof.update({"bound": "alu", "achieved": round(ach_b, 2), "unit": "Gbutterfly/s",
                     "peak": round(peak_b, 2), "frac": round(ach_b / peak_b, 4),
                     "peak_source": "derived: %d SMs x 4 fmaheavy pipes x %.0f MHz x 32 / "
                                    "%.1f pipe cycles per warp-butterfly (ncu, probe)" %
                                    (NUM_SMS, clk_mhz, FMAHEAVY_CYCLES_PER_WARP_BFLY),
                     "probe_gbfly": round(probe / 1e9, 2),
                     # DRAM bytes per limb transform (both passes) from the ncu
                     # capture of the 3072-limb batch (profiles/), against the
                     # algorithmic 1 MiB (each residue read and written once)
                     "traffic": (NTT_DRAM_BYTES_PER_LIMB
                                 if W["logN"] == 16 and tuned[0] == 4 else None),
                     "traffic_unit": "bytes per limb transform (dram read + write, ncu)",
                     "traffic_algorithmic": (1 << W["logN"]) * 8 * 2,
                     "hbm_view": {"achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                                  "frac": round(achieved / hbm, 4)}})
    h2d = sum(host[nm].numel() * 8 for nm in host)
    d2h = 2 * W["k"] * 8
    out = {
        "metric": METRIC if W is WORKLOAD else
        "encrypted-GWAS SNPs/s (245 samples, N=2^17, kappa=3)",
        "value": round(value, 1), "unit": "SNPs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 3),
        "ms_steps": [round(float(x), 3) for x in ms],
        "higher_is_better": True, "scaling": "strong" if shard else "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": W["name"], "N": 1 << W["logN"], "q_limbs": W["L"],
                   "special_primes": W["K"], "dnum": W["dnum"], "n": W["n"], "d": W["d"],
                   "k": W["k"], "kappa": W["kappa"], "layout": layout_used,
                   "parallelism": ("one job sharded by SNP-batch ranges (rank 0 fits, one "
                                   "broadcast of the batch-invariant state, one all-gather)"
                                   if shard else "independent jobs per GPU"),
                   "l2": "flushed between steps (256 MiB write)",
                   "dupm_host_tier_chunk": args.host_state},
        "keyswitch_per_s": round(ks_all / (step_ms / 1e3), 1),
        "keyswitches_per_job": ks_per_job,
        "e2e": {"value": round(snps / (e2e_ms / 1e3), 1), "unit": "SNPs/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": round(e2e_ms, 3)},
        "gpu_launches": int(launches),
        "phases_ms": phases,
        "autotune": {"ntt_shape": tuned[0], "ms_per_shape": tuned[1],
                     "ntt_shape_small": tuned_small[0], "ms_per_shape_small": tuned_small[1]},
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if mccp:
        out["mccp"] = mccp
    if not args.no_micro:
        out["micro"] = run_micro(stream, clk_mhz=clk_mhz, ntt_shape=args.ntt_shape)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(W, layout_used == "factored", ks_hist,
                                           gpu=(data, A, num, den))
    print(json.dumps(out))
    sys.stdout.flush()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


MICRO = dict(name="ntt-ks-micro", logN=16, L=24, q0_bits=60, scale_bits=45, K=8, sp_bits=60,
             dnum=3, n_ct=64, seed=1003)


def keyswitch_work(logN, l, K, alpha):
    """Algorithmic work of one rotation (hybrid key switch) at level l with K
    special primes followed by a rescale: limb transforms (ModUp: the inverse
    transform of c1 and the forward transforms of each digit's new limbs;
    ModDown: inverse of the 2K special limbs, forward of the 2l converted
    limbs; the rescale's inverse of the two last limbs and forward of the
    2(l-1) reduced ones), their butterflies, and the minimum HBM bytes (the
    input and output ciphertexts once, every key byte once)."""
    N = 1 << logN
    beta = -(-l // alpha)
    digits = [min(alpha, l - j * alpha) for j in range(beta)]
    rows_ks = l + sum(l + K - dj for dj in digits) + 2 * K + 2 * l
    rows_rs = 2 + 2 * (l - 1)
    rows = rows_ks + rows_rs
    limbs = 2 * l + 2 * beta * (l + K) + 2 * (l - 1)
    return {"limb_transforms": rows, "ks_limb_transforms": rows_ks,
            "butterflies": rows * (N // 2) * logN,
            "hbm_bytes": limbs * 8 * N, "key_bytes": 2 * beta * (l + K) * 8 * N}


def run_micro(ctx_stream, reps=3, clk_mhz=2070.0, ntt_shape=-1):
    """Kernel microbench: a batched negacyclic NTT + inverse NTT over 64
    ciphertexts x 2 polys x 24 limbs (3072 limb transforms, N = 2^16), and 512
    rotations (64 ciphertexts x steps 1, 2, ..., 128) at level 24, each
    followed by a rescale, run as eight batched sets of 64 (the set path the
    job uses); their roofline against HBM and the butterfly ceiling."""
    import torch
    from paper_1902_04303_gb300 import gwhe
    from paper_1902_04303_gb300.datagen import make_slots
    W = MICRO
    stream = ctx_stream
    ev = _event_maker(stream)
    ctx = gwhe.Context(W["logN"], W["L"], W["q0_bits"], W["scale_bits"], W["K"], W["sp_bits"],
                       W["dnum"], seed=W["seed"], stream=stream.cuda_stream)
    tuned = ctx.autotune()
    ctx.autotune(rows=32)
    if ntt_shape >= 0:
        ctx.set_ntt_variant(ntt_shape)
        tuned = (ntt_shape, tuned[1])
    nvtx = torch.cuda.nvtx
    steps = [1 << i for i in range(8)]
    N, L, nct = ctx.N, W["L"], W["n_ct"]
    rows = nct * 2 * L
    g = torch.Generator(device="cuda")
    g.manual_seed(W["seed"])
    x = torch.empty((nct * 2, L, N), dtype=torch.int64, device="cuda")
    for i in range(L):
        x[:, i, :] = torch.randint(0, ctx.q[i], (nct * 2, N), device="cuda", generator=g)
    ref = x.clone()
    ctx.ntt_batch(x, nct * 2, L)
    ctx.ntt_batch(x, nct * 2, L, inverse=True)
    torch.cuda.synchronize()
    ok = bool(torch.equal(x, ref))
    ms = []
    # NVTX ranges name the timed work, so that profilers can select it
    # (ncu --nvtx --nvtx-include "ntt_3072/")
    for _ in range(reps):
        nvtx.range_push("ntt_3072")
        e0 = ev()
        ctx.ntt_batch(x, nct * 2, L)
        ctx.ntt_batch(x, nct * 2, L, inverse=True)
        e1 = ev()
        nvtx.range_pop()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1) / 2)  # per transform direction
    t_ntt = min(ms) / 1e3
    del x, ref
    probe, probe_ms = ctx.probe_butterflies()
    # batched encoding of 245 REP-like slot vectors (one SNP batch)
    zb = torch.randint(0, 3, (245, ctx.M, 2), device="cuda", generator=g).to(torch.float64)
    ob = torch.empty((245, N), dtype=torch.int64, device="cuda")
    ctx.encode_batch(zb, 245, ctx.delta, ob)
    ems = []
    for _ in range(reps):
        e0 = ev()
        ctx.encode_batch(zb, 245, ctx.delta, ob)
        e1 = ev()
        e1.synchronize()
        ems.append(e0.elapsed_time(e1))
    t_enc = min(ems) / 1e3
    del zb, ob
    ctx.keygen(rot_steps=steps + [3, 5, 6, 7], conj=False)
    # hoisted rotation sums (one ladder group of three doubling steps: rotations
    # 1..7): 210 ciphertexts at 5 limbs (an SNP-batch chunk) and 5 at 20 limbs
    # (a covariate-phase set)
    hoist = {}
    for cnt, lv in ((210, 5), (5, 20)):
        src = [ctx.encrypt(make_slots(ctx.M, 900 + i), ctx.delta, lv, 0x900 + i) for i in range(cnt)]
        outs = ctx.rotate_sum_batch(src, [1, 2, 3, 4, 5, 6, 7])
        hm = []
        for _ in range(reps):
            nvtx.range_push("hoist7_%dx%d" % (cnt, lv))
            e0 = ev()
            ctx.rotate_sum_batch(src, [1, 2, 3, 4, 5, 6, 7], outs)
            e1 = ev()
            nvtx.range_pop()
            e1.synchronize()
            hm.append(e0.elapsed_time(e1))
        hoist["hoisted7_ms_%dx%dlimbs" % (cnt, lv)] = round(min(hm), 3)
        for c_ in src + outs:
            c_.close()
    # 512 rotations + rescales at level 24 as eight sets of 64 ciphertexts
    cts = [ctx.encrypt(make_slots(ctx.M, 7 + i), ctx.delta, L, 0x500 + i) for i in range(nct)]
    outs = [ctx.ct(2, L) for _ in range(nct)]
    for r in steps:
        ctx.rotate_batch(cts, r, rescale=True, outs=outs)
    torch.cuda.synchronize()
    ks = []
    for _ in range(reps):
        nvtx.range_push("ks_level24")
        e0 = ev()
        for r in steps:
            ctx.rotate_batch(cts, r, rescale=True, outs=outs)
        e1 = ev()
        nvtx.range_pop()
        e1.synchronize()
        ks.append(e0.elapsed_time(e1))
    t_ks = min(ks) / 1e3
    ctx.prof_enable(True)
    for r in steps:
        ctx.rotate_batch(cts, r, rescale=True, outs=outs)
    kprof = ctx.prof_read()
    ctx.prof_enable(False)
    # the same 512 one ciphertext at a time (the single-ciphertext entry point)
    torch.cuda.synchronize()
    e0 = ev()
    for c in cts:
        for r in steps:
            o = ctx.rotate(c, r)
            ctx.rescale(o)
            o.close()
    e1 = ev()
    e1.synchronize()
    t_single = e0.elapsed_time(e1) / 1e3
    nrot = nct * len(steps)
    K24, _ = ctx.ks_special(L)
    wk = keyswitch_work(W["logN"], L, K24, -(-L // W["dnum"]))
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    alu = alu_peak_gbfly(clk_mhz)
    t_hbm = nrot * wk["hbm_bytes"] / (hbm * 1e9)
    t_alu = nrot * wk["butterflies"] / (alu * 1e9)
    kern_ms = sum(v[0] for v in kprof.values())
    ks_roof = {
        "op": "rotation (hybrid key switch, K_l = %d special primes) + rescale at level %d"
              % (K24, L),
        "count": nrot, "ms": round(t_ks * 1e3, 3), "kernel_ms": round(kern_ms, 3),
        "per_s": round(nrot / t_ks, 1),
        "per_op": wk,
        "hbm": {"achieved_gbs": round(nrot * wk["hbm_bytes"] / t_ks / 1e9, 1), "peak": hbm,
                "frac": round(t_hbm / t_ks, 4)},
        "alu": {"achieved_gbfly": round(nrot * wk["butterflies"] / t_ks / 1e9, 2),
                "peak": round(alu, 2), "frac": round(t_alu / t_ks, 4)},
        "bound": "alu" if t_alu >= t_hbm else "hbm",
        "frac": round(max(t_alu, t_hbm) / t_ks, 4),
        "classes": class_rates(kprof),
        "one_at_a_time_ms": round(t_single * 1e3, 2),
        "one_at_a_time_per_s": round(nrot / t_single, 1)}
    for c_ in cts + outs:
        c_.close()
    return {"workload": W["name"], "ntt_roundtrip_exact": ok,
            "ntt_shape": tuned[0], "ntt_ms_per_shape_512_rows": tuned[1],
            "ntt_limb_per_s": round(rows / t_ntt, 1),
            "ntt_gbs_algorithmic": round(rows * N * 16 / t_ntt / 1e9, 1),
            "ntt_ms_3072_limbs": round(t_ntt * 1e3, 3),
            "ntt_gbfly_per_s": round(rows * (N // 2) * W["logN"] / t_ntt / 1e9, 2),
            "ntt_alu_frac": round(rows * (N // 2) * W["logN"] / t_ntt / 1e9 / alu, 4),
            "probe_gbfly_per_s": round(probe / 1e9, 2), "probe_ms": round(probe_ms, 3),
            "encode_ms_245": round(t_enc * 1e3, 3),
            "rotations": nrot,
            "keyswitch_per_s_level24": ks_roof["per_s"],
            "keyswitch_roofline": ks_roof, **hoist}


def oracle_sample(W, levels=(4,), threads=1):
    """Times the CPU oracle on one key switch at each given level (random
    input and random keys of the family that level uses: the oracle's cost
    does not depend on the values), and one tensor and one encryption at the
    SNP-batch level (4 limbs), with `threads` host threads."""
    from oracle.ckks import Ct, OracleCKKS, lib
    lib().or_set_threads(threads)
    o = OracleCKKS(logN=W["logN"], L=W["L"], q0_bits=W["q0_bits"], scale_bits=W["scale_bits"],
                   K=W["K"], sp_bits=W["sp_bits"], dnum=W["dnum"], seed=W["seed"])
    rng = np.random.Generator(np.random.PCG64(5))
    N = o.N

    def rnd(lv, npoly):
        return Ct(np.stack([np.stack([rng.integers(0, o.q[i], size=N, dtype=np.uint64)
                                      for i in range(lv)]) for _ in range(npoly)]), o.delta)

    t0 = time.perf_counter()
    o.pk_b = rnd(W["L"], 1).c[0]
    o.pk_a = rnd(W["L"], 1).c[0]
    fams = {}
    for l in levels:
        k = o.ks_k[l]
        if k not in fams:
            lmax = o.key_lmax[k]
            fams[k] = rng.integers(0, 2 ** 59, size=(-(-lmax // o.alpha), 2, lmax + k, N),
                                   dtype=np.uint64)
    o.keys[0] = fams
    t_setup = time.perf_counter() - t0
    t_ks = {}
    for l in levels:
        x = rnd(l, 1).c[0]
        t0 = time.perf_counter()
        o.keyswitch(x, 0)
        t_ks[l] = time.perf_counter() - t0
    a, b = rnd(4, 2), rnd(4, 2)
    t0 = time.perf_counter()
    o.tensor(a, b)
    t_tensor = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.encrypt(rnd(4, 1).c[0], 1, o.delta)
    t_enc = time.perf_counter() - t0
    used = lib().or_get_threads()
    lib().or_set_threads(os.cpu_count() or 1)
    return dict(t_ks=t_ks, t_tensor4=t_tensor, t_enc4=t_enc, t_setup=t_setup, alpha=o.alpha,
                ks_k=list(o.ks_k), threads=used)


def extrapolate(sample, ks_hist, W, factored=False):
    """Oracle job time: each level's key switches at that level's measured
    cost (a level without its own sample: the nearest sampled level, scaled by
    the polynomial-product count 2 beta (l + K_l) of a switch), plus the
    batches' tensor products and SNP encryptions (M-CCP: n of each at 4
    limbs; factored: one encryption at 6 limbs, d tensors at 6 and d at 4
    limbs, scaled by limbs).  A hoisted ladder group counts as one switch, so
    this is a lower bound on the oracle's time."""
    alpha, ks_k, t_ks = sample["alpha"], sample["ks_k"], sample["t_ks"]

    def work(l):
        return math.ceil(l / alpha) * (l + ks_k[l])

    t = 0.0
    for l, cnt in enumerate(ks_hist):
        if not cnt:
            continue
        ref = l if l in t_ks else min(t_ks, key=lambda s: abs(s - l))
        t += cnt * t_ks[ref] * work(l) / work(ref)
    tau = 2 * ((1 << (W["logN"] - 1)) // (1 << math.ceil(math.log2(W["n"]))))
    batches = -(-W["k"] // tau)
    if factored:
        t += batches * (sample["t_enc4"] * 6 / 4
                        + W["d"] * sample["t_tensor4"] * (6 / 4 + 1))
    else:
        t += batches * W["n"] * (sample["t_tensor4"] + sample["t_enc4"])
    return t


def accuracy_report(data, A, num, den, kappa):
    """The timed job's decrypted statistics against the plaintext FP64 run of
    the same approximated GWAS (the parity tolerances |d b'| <= 5e-3 and
    |d(-log10 p)| <= 0.05), and the paper's accuracy report against the
    exact semi-parallel method (section Results: the number of -log10 p
    values that differ by more than e, and the least-squares line of b' on
    b), with the time of the FP64 run."""
    from oracle import gwas_exact, gwas_fp64
    t0 = time.perf_counter()
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=kappa, A=A)
    t_fp64 = time.perf_counter() - t0
    ok = np.abs(ref["den"]) > 1e-6  # monomorphic SNPs have den = 0
    b = num[ok] / den[ok]
    lp = gwas_fp64.neglog10p(b, 1.0 / den[ok])
    db = float(np.max(np.abs(b - ref["b"][ok])))
    dl = float(np.max(np.abs(lp - gwas_fp64.neglog10p(ref["b"][ok], ref["err"][ok]))))
    ex = gwas_exact.semi_parallel_exact(data.X, data.y, data.S)
    lpx = gwas_fp64.neglog10p(ex["b"][ok], ex["err"][ok])
    diff = np.abs(lp - lpx)
    m = int(ok.sum())
    counts = {("%g" % e): {"entries": int(np.sum(diff > e)),
                           "accuracy_pct": round(100.0 * (1 - np.sum(diff > e) / m), 2)}
              for e in (0.1, 0.01, 0.005)}
    slope, icpt = np.polyfit(ex["b"][ok], b, 1)
    return ({"ms": round(t_fp64 * 1e3, 1), "max_abs_db": db, "max_abs_dlog10p": dl,
             "within_tolerance": bool(db <= 5e-3 and dl <= 0.05), "snps": m},
            {"vs": "exact semi-parallel GWAS (exact sigmoid, converged Newton, W-weighted)",
             "abs_dlog10p_above": counts, "polyfit_b_enc_on_b_exact":
                 {"slope": round(float(slope), 5), "intercept": round(float(icpt), 7)}})


def cpu_baseline(W, factored, ks_hist, gpu=None):
    """The oracle on a bounded sample of the job, on all host cores and on one
    thread, extrapolated with the job's key-switch histogram; with gpu =
    (data, A, num, den) also the plaintext FP64 GWAS of the same inputs and
    the accuracy report of the timed job."""
    cores = os.cpu_count() or 1
    levels = [l for l, c in enumerate(ks_hist) if c]
    s_all = oracle_sample(W, levels=levels, threads=cores)
    s_one = oracle_sample(W, levels=(4,), threads=1)
    t_all = extrapolate(s_all, ks_hist, W, factored)
    t_one = extrapolate(s_one, ks_hist, W, factored)
    out = {"value": round(W["k"] / t_all, 4), "unit": "SNPs/s", "cores": s_all["threads"],
           "kind": "oracle", "nproc": cores,
           "single_thread": {"value": round(W["k"] / t_one, 4), "cores": 1,
                             "s_per_job": round(t_one, 1)},
           "s_per_job": round(t_all, 1),
           "sample": ("oracle timed on one key switch at each of the %d levels the job switches "
                      "at (%.1f s in all, %d threads) and one tensor and one encryption at 4 "
                      "limbs, N=2^%d; extrapolated to the job with its key-switch histogram "
                      "(%d switches, %s layout) and the batches' tensors/encryptions: %.0f s per "
                      "job (extrapolated; one thread: %.0f s from a level-4 sample)"
                      % (len(levels), sum(s_all["t_ks"].values()), s_all["threads"], W["logN"],
                         int(np.sum(ks_hist)), "factored" if factored else "M-CCP", t_all,
                         t_one))}
    if gpu is not None:
        data, A, num, den = gpu
        out["plaintext_fp64"], out["accuracy_vs_exact"] = accuracy_report(data, A, num, den,
                                                                          W["kappa"])
    return out


def run_reference(args):
    """The oracle arm: each step is a bounded sample of the job on the host
    cores (one key switch per level the job switches at), extrapolated to the
    job's SNPs/s with its key-switch histogram."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W = BENCH_WORKLOADS.get(args.workload, WORKLOAD)
    from oracle import build_oracle
    build_oracle.build()
    from oracle.trace import job_ks_histogram
    # the same SNP-phase layout as the library arm (auto: factored when the
    # ring has more than 8 limbs)
    factored = args.layout == "factored" or (args.layout == "auto" and W["L"] > 8)
    # key switches per level of the job, from a level trace of the oracle circuit
    hist, _, _ = job_ks_histogram(W, W["kappa"], factored)
    levels = [l for l, c in enumerate(hist) if c]
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_sample(W, levels=(4,), threads=cores)
    # step i times one key switch at level levels[i mod #levels] (and the
    # batch-level tensor and encryption); the job time is extrapolated from
    # all the steps' samples together
    merged = None
    t_all = time.perf_counter()
    for i in range(args.steps):
        s = oracle_sample(W, levels=(levels[i % len(levels)],), threads=cores)
        if merged is None:
            merged = s
        else:
            merged["t_ks"].update(s["t_ks"])
            for key in ("t_tensor4", "t_enc4"):
                merged[key] = min(merged[key], s[key])
    wall = time.perf_counter() - t_all
    used = merged["threads"]
    t_job = extrapolate(merged, hist, W, factored)
    value = W["k"] / t_job
    out = {"metric": METRIC if W is WORKLOAD else
           "encrypted-GWAS SNPs/s (245 samples, N=2^17, kappa=3)",
           "value": round(value, 4), "unit": "SNPs/s", "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_job * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": W["name"], "N": 1 << W["logN"], "q_limbs": W["L"],
                      "special_primes": W["K"], "dnum": W["dnum"], "n": W["n"], "d": W["d"],
                      "k": W["k"], "kappa": W["kappa"],
                      "layout": "factored" if factored else "mccp"},
           "cpu_baseline": {"value": round(value, 4), "unit": "SNPs/s", "cores": used,
                            "kind": "oracle",
                            "sample": "per step: one key switch at one of the %d levels the job "
                                      "switches at (in turn), one tensor and one encryption at 4 "
                                      "limbs, N=2^%d, on %d threads; the job extrapolated from "
                                      "the %d samples (%.1f s wall)"
                                      % (len(levels), W["logN"], used, len(merged["t_ks"]),
                                         wall)},
           "e2e": {"value": round(value, 4), "unit": "SNPs/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ------------------------------------------------------------ cohorts / serving
COHORTS = dict(name="cohorts16", logN=16, L=24, q0_bits=60, scale_bits=45, K=8, sp_bits=60,
               dnum=3, jobs=16, seed=1004, kappa=1)
SERVING = dict(name="serving", requests=200, big_fraction=0.05, big=(6000, 4, 100000), seed=1005)


def cohort_shapes(count, seed):
    """uneven cohorts: n ~ U{100..1000}, d ~ U{2..6} (with the intercept),
    k ~ U{1000..50000}, seeded"""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [(int(rng.integers(100, 1001)), int(rng.integers(2, 7)), int(rng.integers(1000, 50001)))
            for _ in range(count)]


def _serving_ctx(gwhe, stream, shapes):
    W = COHORTS
    ctx = gwhe.Context(W["logN"], W["L"], W["q0_bits"], W["scale_bits"], W["K"], W["sp_bits"],
                       W["dnum"], seed=W["seed"], stream=stream.cuda_stream)
    steps = []
    for n, d, k in set(shapes):
        job = gwhe.Job(ctx, n, d, k)
        steps += [r for r in job.rotation_steps() if r not in steps]
        job.close()
    ctx.keygen(rot_steps=steps, conj=True)
    ctx.autotune()
    ctx.autotune(rows=32)
    return ctx


def _cohort_inputs(shapes, seed):
    from paper_1902_04303_gb300.datagen import make_gwas
    out = []
    for i, (n, d, k) in enumerate(shapes):
        data = make_gwas(n, d, k, seed=seed + i)
        out.append((data, client_preprocess(data.X)))
    return out


def run_cohorts(args):
    """Batched uneven cohorts: 16 jobs one at a time on one stream, then all
    submitted at once to the serving engine (workers with their own streams
    sharing the keys); total SNPs / wall time for both."""
    import torch
    from paper_1902_04303_gb300 import build as pkg_build
    from paper_1902_04303_gb300 import gwhe
    pkg_build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    W = COHORTS
    shapes = cohort_shapes(W["jobs"], W["seed"])
    ctx = _serving_ctx(gwhe, stream, shapes)
    inputs = _cohort_inputs(shapes, W["seed"] + 100)
    snps = sum(k for _, _, k in shapes)

    def one(i):
        (data, A) = inputs[i]
        n, d = data.X.shape
        job = gwhe.Job(ctx, n, d, data.S.shape[1])
        job.set_nonce(i + 1)
        job.encrypt_inputs(data.X, A, data.y)
        job.fit(W["kappa"])
        job.snp_stats(data.S)
        r = job.decrypt_results()
        job.close()
        return r

    one(0)  # warm-up: tables, caches, the memory pool
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = [one(i) for i in range(len(shapes))]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    srv = gwhe.Server(ctx, workers=args.workers, chunk_batches=64,
                      one_snp_loop=args.one_snp_loop)
    t0 = time.perf_counter()
    ids = [srv.submit(data.X, A, data.y, data.S, kappa=W["kappa"], nonce=i + 1, borrow=True)
           for i, (data, A) in enumerate(inputs)]
    res = [srv.wait(rid) for rid in ids]
    t_srv = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    same = all(np.array_equal(a[0], b[0], equal_nan=True) and
               np.array_equal(a[1], b[1], equal_nan=True) for a, b in zip(seq, res))
    out = {"metric": "batched uneven-cohort encrypted-GWAS SNPs/s (16 jobs, N=2^16)",
           "value": round(snps / t_srv, 1), "unit": "SNPs/s", "n_gpus": 1, "steps": 1,
           "warmup": 1, "ms_per_step": round(t_srv * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": W["name"], "jobs": [list(x) for x in shapes],
                      "workers": args.workers, "snps": snps,
                      "one_snp_loop_at_a_time": bool(args.one_snp_loop)},
           "one_at_a_time": {"value": round(snps / t_seq, 1), "ms": round(t_seq * 1e3, 1)},
           "speedup_vs_one_at_a_time": round(t_seq / t_srv, 3),
           "same_results_alone_and_batched": bool(same),
           "peak_bytes_claimed": st["peak_bytes_claimed"]}
    print(json.dumps(out))


def run_serving(args):
    """Serving: Poisson arrivals of GWAS requests (the cohort mix plus a few
    6000 x 100000 jobs), admitted by HBM footprint as workers and memory
    free up; p50/p99 latency beside SNPs/s."""
    import threading

    import torch
    from paper_1902_04303_gb300 import build as pkg_build
    from paper_1902_04303_gb300 import gwhe
    pkg_build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    S_ = SERVING
    nreq = args.requests
    t_setup = time.perf_counter()

    def progress(msg):  # a trace on stderr of where a long run stands
        print("[serving %.0f s] %s" % (time.perf_counter() - t_setup, msg), file=sys.stderr,
              flush=True)

    rng = np.random.Generator(np.random.PCG64(S_["seed"]))
    mix = cohort_shapes(nreq, S_["seed"] + 1)
    shapes = [S_["big"] if rng.random() < S_["big_fraction"] else mix[i] for i in range(nreq)]
    ctx = _serving_ctx(gwhe, stream, shapes)
    progress("keys and tables ready")
    inputs = _cohort_inputs(shapes, S_["seed"] + 1000)
    progress("inputs of %d requests generated" % nreq)
    srv = gwhe.Server(ctx, workers=args.workers, chunk_batches=64,
                      one_snp_loop=args.one_snp_loop)
    # calibration: service time t = a + b u of 4 jobs of the mix, one at a time,
    # against the key switches of their SNP batches u (batches x switches per
    # batch of the factored layout); the mean service over all requests
    # (the big jobs included) from the fit sets the rate for ~80 % load
    def units(n, d, k):
        nb = 1 << int(math.ceil(math.log2(n)))
        tau = 2 * ((1 << 15) // nb)
        h = -(-int(math.log2(nb)) // 3)
        return -(-k // tau) * (d + 2 * d * h + 6 + 3 * h)

    cal, cu = [], []
    for i in range(min(4, nreq)):
        data, A = inputs[i]
        t0 = time.perf_counter()
        srv.wait(srv.submit(data.X, A, data.y, data.S, nonce=4000 + i))
        cal.append(time.perf_counter() - t0)
        cu.append(units(*shapes[i]))
    b, a = np.polyfit(cu, cal, 1) if len(set(cu)) > 1 else (float(np.mean(cal)) / cu[0], 0.0)
    a, b = max(float(a), 0.0), max(float(b), 1e-9)
    mean_service = a + b * float(np.mean([units(*x) for x in shapes]))
    rate = 0.8 / mean_service if args.rate <= 0 else args.rate  # ~80% busy
    progress("calibrated: %.3f s mean service, %.3f arrivals/s" % (mean_service, rate))
    gaps = rng.exponential(1.0 / rate, size=nreq)
    lat = [None] * nreq
    lock = threading.Lock()
    done = [0]

    def waiter(i, rid):
        _, _, t = srv.wait(rid)
        with lock:
            lat[i] = t
            done[0] += 1
            if done[0] % 20 == 0:
                progress("%d of %d requests done, server %s" % (done[0], nreq, srv.stats()))

    threads = []
    t0 = time.perf_counter()
    t_next = t0
    for i in range(nreq):
        t_next += gaps[i]
        dt = t_next - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        data, A = inputs[i]
        rid = srv.submit(data.X, A, data.y, data.S, nonce=i + 1, borrow=True)
        th = threading.Thread(target=waiter, args=(i, rid))
        th.start()
        threads.append(th)
    for th in threads:
        th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    tot = np.array([x["latency_ms"] for x in lat])
    big = np.array([x == S_["big"] for x in shapes])
    snps = sum(k for _, _, k in shapes)
    out = {"metric": "served encrypted-GWAS SNPs/s with p50/p99 latency (Poisson arrivals, N=2^16)",
           "value": round(snps / wall, 1), "unit": "SNPs/s", "n_gpus": 1, "steps": 1, "warmup": 0,
           "ms_per_step": round(wall * 1e3, 1), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": "serving%d" % nreq, "requests": nreq,
                      "big_jobs": sum(1 for x in shapes if x == S_["big"]),
                      "arrival_rate_per_s": round(rate, 3), "workers": args.workers,
                      "one_snp_loop_at_a_time": bool(args.one_snp_loop)},
           "latency_ms": {"p50": round(float(np.percentile(tot, 50)), 1),
                          "p99": round(float(np.percentile(tot, 99)), 1),
                          "max": round(float(tot.max()), 1)},
           "latency_ms_cohort_mix": {
               "p50": round(float(np.percentile(tot[~big], 50)), 1),
               "p99": round(float(np.percentile(tot[~big], 99)), 1)},
           "latency_ms_big_jobs": ({"p50": round(float(np.percentile(tot[big], 50)), 1),
                                    "max": round(float(tot[big].max()), 1)}
                                   if big.any() else None),
           "mean_service_s_estimated": round(mean_service, 3),
           "queue_ms_p50": round(float(np.percentile([x["queue_ms"] for x in lat], 50)), 1),
           "peak_bytes_claimed": st["peak_bytes_claimed"], "budget_bytes": st["budget"]}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gwhe", choices=["gwhe", "reference"])
    ap.add_argument("--layout", default="auto", choices=["auto", "mccp", "factored"],
                    help="SNP-phase layout: S' = M S with M as a CCP matrix, or the "
                         "factored S' = S - XA(X^T S) with S in CCP")
    ap.add_argument("--host-state", type=int, default=0,
                    help="M-CCP layout: keep Dup(M_j) in pinned host memory, prefetched this "
                         "many columns at a time (0: on the device)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-micro", action="store_true")
    ap.add_argument("--no-mccp", action="store_true",
                    help="skip the M-CCP layout's timing beside the factored headline")
    ap.add_argument("--micro-only", action="store_true",
                    help="only the kernel microbench (the controlled case for profiler captures)")
    ap.add_argument("--workload", default="paper-n245",
                    choices=["paper-n245", "paper-n245-kappa3", "cohorts16", "serving"],
                    help="paper-n245: the paper-shaped job; paper-n245-kappa3: the same at "
                         "N=2^17 with kappa=3; cohorts16: 16 uneven cohorts one at a time and "
                         "batched; serving: Poisson request stream")
    ap.add_argument("--workers", type=int, default=4, help="serving-engine workers")
    ap.add_argument("--shard-job", action="store_true",
                    help="with --gpus N: shard one job over the ranks (strong scaling) instead of "
                         "one independent job per GPU")
    ap.add_argument("--one-snp-loop", action="store_true",
                    help="serving engine: SNP loops one at a time at high priority, covariate "
                         "phases overlapping them at low priority")
    ap.add_argument("--ntt-shape", type=int, default=-1,
                    help="use this compiled shape of the N=2^16 transform for every launch "
                         "instead of the autotuned ones (for profiler captures)")
    ap.add_argument("--requests", type=int, default=SERVING["requests"])
    ap.add_argument("--rate", type=float, default=0.0, help="arrivals/s (0: ~80%% busy)")
    args = ap.parse_args()
    if args.impl != "reference" and args.workload == "cohorts16":
        run_cohorts(args)
        return
    if args.impl != "reference" and args.workload == "serving":
        run_serving(args)
        return
    if args.micro_only:
        import torch
        from paper_1902_04303_gb300 import build as pkg_build
        pkg_build.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(run_micro(torch.cuda.current_stream(), reps=max(1, args.steps),
                                   ntt_shape=args.ntt_shape)))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
