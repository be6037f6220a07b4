"""Benchmark of the hot path on one GB300 (or N, one process per GPU).

Workload (default): 2-D periodic image 256x256, db4 (8 taps), L = 4 levels, m = 16 terms
(4x4 bilinear hat windows), 15x15 Gaussian kernels sigma_k = 0.5 + 2.5 k/15, pattern
| |mu| - |lambda| | <= 2 with the support rule (nnz = 123,896,832).  One step is one pass
of the whole hot path:
  pc_assemble  (FP64 base wavelets, filtered wavelets, fused window-multiply + localized
                transform, FP32 Theta + BF16 copy)
  pc_apply     (y = Theta x, 16 right-hand sides, BF16 Theta, FP32 accumulation)
  pc_backward  (dL/du, dL/dv for L = 1/2 ||Theta||^2, i.e. dL/dTheta = Theta)
`value` = Theta entries per second of the whole step (nnz / step time, summed over ranks).
The end of the line summarises the metric's own numbers: the batched FP32 assembly of 64
uneven operators against the plain FP64 assembly of each (`batch_c4`), the large 1024^2
workload (`c5_1024`: assembly, BF16 apply to 16 right-hand sides, backward), the single-operator
FP32 vs FP64 assembly (`assembly_c2`), every result's error against the FP64 oracle
(`errors_vs_oracle`) and the backward time (`bwd_ms`).

--impl reference times the FP64 CPU oracle (the paper's Algorithm 2) on the machine's host
cores, on a bounded sample of columns of the same workload, in the same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Theta entries/s + HBM GB/s, batched FP32 vs plain FP64 on 1 GB300 @1e-5; bwd ms"
UNIT = "Theta entries/s"
WORKLOAD = ("c2: 2-D periodic 256x256, db4 J=4, m=16 (4x4 bilinear hats), 15x15 Gaussians "
            "sigma 0.5->3, pattern |j-j'|<=2 + support distance <= kernel radius; step = "
            "assemble (FP32 Kahan + BF16 copy) + apply (16 RHS, BF16) + backward")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------- algorithmic FP32 work of stage 1 (the second roofline: the FP32 pipe) ----------------
# FP32 peak derived from the unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _cdiv(a, b):
    return -((-a) // b)


def _wlen(j, Lf):
    return ((1 << j) - 1) * (Lf - 1) + 1


def _woff(j, e, Lf):
    return (1 << (j - 1)) * (2 - Lf) if e else 0


def _rng_cascade(lo, cnt, full, Lf, nout):
    # union of the low- and high-pass output ranges of one cascade step (taps [0, Lf-1], [2-Lf, 1])
    nlo = _cdiv(lo - Lf + 1, 2)
    c = (lo + cnt - 1 + Lf - 2) // 2 - nlo + 1
    return (nlo, nout, 1) if (full or c >= nout) else (nlo, c, 0)


def _rng_filter(lo, cnt, full, S, ln, nout):
    nlo = _cdiv(lo - ln + 1, S)
    c = (lo + cnt - 1) // S - nlo + 1
    return (nlo, nout, 1) if (full or c >= nout) else (nlo, c, 0)


def assembly_flops(op, phases=8):
    """Algorithmic FP32 operations of one 2-D assembly (no compensation terms counted): the
    window-weighted sums (a multiply and an add per nonzero window of each region pixel) and the
    localized transforms (per output position of a level, both filters: 4 Lf flops per line of
    the union output range), averaged over `phases` translates per axis of every band."""
    n, L, Lf, r, gap = op.n, op.levels, 2 * op.delta, op.r, op.gap
    nzw = float(np.mean((np.asarray(op.v) != 0).sum(axis=0)))   # nonzero windows per pixel
    bands = [(L, 0, 0)] + [(j, e0, e1) for j in range(L, 0, -1) for (e0, e1) in ((0, 1), (1, 0), (1, 1))]
    total = 0.0
    for (j, e0, e1) in bands:
        nj = n >> j
        jlo = 1 if gap < 0 else max(1, j - gap)
        jhi = L if gap < 0 else min(L, j + gap)
        k0 = jlo - 1
        lenk = _wlen(k0, Lf) if k0 > 0 else 0
        acc, cnt = 0.0, 0
        for l in range(min(nj, phases)):
            def region(e):
                lo, c = (l << j) + _woff(j, e, Lf) - r, _wlen(j, Lf) + 2 * r
                return (lo, n, 1) if c >= n else (lo, c, 0)
            A0, A1 = region(e0), region(e1)
            f = 2.0 * nzw * A0[1] * A1[1]
            p0, p1 = A0, A1
            for jj in range(1 if k0 == 0 else k0, jhi + 1):
                njj = n >> jj
                if jj == k0:   # LL of level k0 by the sampled scaling function at stride 2^k0
                    q0 = _rng_filter(*A0, 1 << k0, lenk, njj)
                    q1 = _rng_filter(*A1, 1 << k0, lenk, njj)
                    f += 2.0 * lenk * (A0[1] * q1[1] + q1[1] * q0[1])
                else:
                    q0 = _rng_cascade(*p0, Lf, njj)
                    q1 = _rng_cascade(*p1, Lf, njj)
                    f += 4.0 * Lf * (p0[1] * q1[1] + 2 * q1[1] * q0[1])
                p0, p1 = q0, q1
            acc += f
            cnt += 1
        total += acc / cnt * nj * nj
    return total


def _csrc_sha():
    """SHA-256 of the CUDA sources (names and contents), to tell whether a profile still applies."""
    import hashlib
    d = os.path.join(ROOT, "paper_2005_09870_gb300", "csrc")
    hsh = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        hsh.update(f.encode())
        hsh.update(open(os.path.join(d, f), "rb").read())
    return hsh.hexdigest()


def profile_traffic(kernels):
    """DRAM bytes (read + write) per launch of the named kernels of the 256^2 workload, summed,
    from the committed ncu summary profiles/traffic_c2.json; None when that capture was taken on
    other CUDA sources than the ones built now, or is missing."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "traffic_c2.json")))
        if d.get("csrc_sha256") != _csrc_sha():
            return None
        return int(sum(d["kernels"][k]["dram_bytes_per_launch"] for k in kernels))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        out_dir = os.environ.get("PC_BENCH_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(op, seconds, seed=5, max_cols=65536, nthreads=0):
    """Algorithm 2 (FP64 oracle, OpenMP over columns; nthreads 0 = all cores) on uniformly drawn
    columns until about `seconds` of oracle time: returns (entries/s counted on the pattern,
    columns, threads, wall)."""
    import oracle
    rng = np.random.default_rng(seed)
    threads = nthreads if nthreads > 0 else oracle.max_threads()
    batch = max(threads, 8) if nthreads != 1 else 2
    done = entries = 0
    wall = 0.0
    while wall < seconds and done < max_cols:
        cols = rng.integers(0, op.N, size=batch)
        t0 = time.perf_counter()
        oracle.theta_columns(op, cols, nthreads=threads)
        wall += time.perf_counter() - t0
        entries += sum(int(oracle.pattern_column(op, c).sum()) for c in cols)   # untimed
        done += batch
    return entries / wall, done, threads, wall


# ---------------- multi-rank plumbing (one process per GPU, replicas of the workload) ----------------
def rank_workload(name, rank):
    """The rank's replica: the same workload shape with rank-dependent seeds (independent data)."""
    import pc_inputs as P
    return P.workload(name, seed_offset=rank)


def max_over_ranks(x, device, world):
    """Max of a per-rank float over the process group (the slowest rank times the job)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, ms):
    """Weak scaling: every rank processes its own replica; units of all ranks / the max time."""
    return world * units_per_rank / (ms * 1e-3)


def bench_config(world):
    """The `config` of both arms' lines (the same dict, so that the two lines compare)."""
    return {"workload": WORKLOAD, "nrhs": 16, "l2": "flushed between steps (256 MB write, untimed)",
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}


def run_reference(args, rank, world):
    """The oracle arm: FP64 CPU Algorithm 2 on the host cores, rank 0 only.  Loads only the
    oracle's library."""
    if rank != 0:
        return
    import oracle
    import pc_inputs as P
    oracle.build()
    op = P.workload(args.workload)
    rng = np.random.default_rng(7)
    threads = oracle.max_threads()
    ncols = max(threads, 16)
    for _ in range(args.warmup):
        oracle.theta_columns(op, rng.integers(0, op.N, size=ncols))
    times, entries = [], 0
    for _ in range(args.steps):
        cols = rng.integers(0, op.N, size=ncols)
        t0 = time.perf_counter()
        oracle.theta_columns(op, cols)
        times.append(time.perf_counter() - t0)
        entries += sum(int(oracle.pattern_column(op, c).sum()) for c in cols)
    wall = sum(times)
    rate = entries / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(world),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{ncols} uniformly drawn columns per step, Algorithm 2 in FP64"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_fista(pw, g, op, rank, dev, stream, iters):
    """FISTA-W and FISTA-WP iterations (pc_fista) on the FP32 Theta of the bench operator: a
    seeded sparse-plus-noise problem z0, weights 0.02, step 0.95 / (power-iteration norm).  One
    iteration = Theta y - z0 and Theta^T r (both gathers, the second over the transposed copy),
    then the update; the FP32 values (4 bytes x nnz, larger than L2) stream from HBM twice per
    iteration."""
    import torch
    import pc_inputs as P
    N, nnz = op.N, g.nnz
    zt = torch.tensor(P.normal(P.BASE_SEED + 300 + rank, N) * (P.uniform(P.BASE_SEED + 301 + rank, N) < 0.1),
                      dtype=torch.float32, device=dev)
    z0 = torch.empty_like(zt)
    pw.pc_apply(g.h, zt, z0)               # BF16 copy; only makes the data
    z0 += 0.01 * torch.tensor(P.normal(P.BASE_SEED + 302 + rank, N), dtype=torch.float32, device=dev)
    w = torch.full((N,), 0.02, dtype=torch.float32, device=dev)
    out = {"workload": "the bench operator's Theta (FP32 values), one image, sparse + 1% noise, w = 0.02",
           "iters": iters, "l2": "not flushed: Theta's FP32 values exceed L2"}
    peak, peak_kind = _peaks()
    for name, sigma in (("fista_w", None), ("fista_wp", "jacobi")):
        sig = None
        if sigma:
            J = g.jacobi()
            sig = 1.0 / torch.clamp(J, min=1e-30)
        t0 = time.time()
        L = pw.pc_power_norm(g.h, sig, 30)
        pn_ms = (time.time() - t0) * 1e3
        tau = 0.95 / L
        z = torch.zeros(N, dtype=torch.float32, device=dev)
        pw.pc_fista(g.h, z0, w, sig, z, 3, tau)        # warm-up
        z.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        l0 = pw.pc_launch_counter()
        a.record(stream)
        pw.pc_fista(g.h, z0, w, sig, z, iters, tau)
        b.record(stream)
        torch.cuda.synchronize()
        launches = pw.pc_launch_counter() - l0
        g.sync()
        ms_it = a.elapsed_time(b) / iters
        # algorithmic bytes: Theta twice (4 B/entry: the stored values, then the transposed copy),
        # y gathered, z0 read and r written by the first product, r gathered and g written by the
        # second, the update reads z, y, g, w (+ sigma) and writes z, y
        vec = N * 4 * (3 + 2 + 6 + (1 if sig is not None else 0))
        alg = 2 * 4 * nnz + vec
        gbs = alg / (ms_it * 1e-3) / 1e9
        out[name] = {"ms_per_iter": ms_it, "iters_per_s": 1e3 / ms_it, "lipschitz": L, "tau": tau,
                     "power_norm_30_iters_host_ms": pn_ms, "kernel_launches": int(launches),
                     "nnz_per_s": 2 * nnz / (ms_it * 1e-3), "nonzeros_in_z": int((z != 0).sum()),
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                  "frac": gbs / peak, "bytes_per_iter": alg, "peak_kind": peak_kind}}
    return out


def run_sweep(pw, rank, dev, stream, sides=(128, 256, 512, 1024, 2048)):
    """Assembly times of the stand-ins for the paper's two blurs (Section 4.1; Symmlet 6,
    L = 4, op1: m = 5 / 19x19, op2: m = 25 / 25x25) on square images of side 2^7..2^11 (the
    paper's timing sweep goes to 2^12 with its thresholded, much sparser matrix; the exact
    pattern at 2^12 would need ~270 GB for its FP32 values alone).  FP32 Theta, no BF16 copy, CUDA events around
    pc_assemble, inputs larger than L2 from side 256 on."""
    import torch
    import pc_inputs as P
    out = []
    for name in ("op1", "op2"):
        for n in sides:
            rec = {"operator": name, "side": n}
            g = None
            try:
                op = P.workload(name, n=n, seed_offset=rank)
                g = pw.PCOperator(pw.desc_of(op, pw.PC_FP32, 0), torch.tensor(op.u, dtype=torch.float32, device=dev),
                                  torch.tensor(op.v, dtype=torch.float32, device=dev))
                for _ in range(2):
                    g.assemble()
                ts = []
                for _ in range(3):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    g.assemble()
                    b.record(stream)
                    torch.cuda.synchronize()
                    ts.append(a.elapsed_time(b))
                g.sync()
                ms = float(np.median(ts))
                rec.update({"N": op.N, "m": op.m, "stencil": 2 * op.r + 1, "nnz": g.nnz, "assemble_ms": ms,
                            "entries_per_s": g.nnz / (ms * 1e-3),
                            "hbm_gbs_algorithmic": (4 * g.nnz + 4 * op.m * op.N) / (ms * 1e-3) / 1e9})
            except Exception as e:                  # recorded, not fatal to the bench line
                rec["error"] = str(e)[:200]
            finally:
                if g is not None:
                    try:
                        g.close()
                    except Exception:
                        pass
            out.append(rec)
    return out


# The paper's Algorithm 1 decomposition times in seconds (FP64 on a 12-core CPU, eta = 5e-4,
# Symmlet 6; the timing-vs-N figure of Section 4.2), for context beside the GPU's.
PAPER_ALG1_S = {"op1": {128: 3.35, 256: 15.7, 512: 78.3, 1024: 430.9, 2048: 2292.0, 4096: 13048.0},
                "op2": {128: 14.9, 256: 72.6, 512: 345.8, 1024: 1816.6, 2048: 9747.7, 4096: 56192.9}}


def run_alg1(pw, rank, dev, check, sides=(128, 256, 512, 1024), discard_sides=(2048, 4096), ops=("op1", "op2"),
             vs_eta=True, eta=5e-4):
    """Thresholded Algorithm 1 on the GPU (pc_alg1_create, Section 3.2) on the stand-ins for the
    paper's two blurs: eta = 5e-4 with the plain cut tau_k = eps_k, FP32 products, sides
    2^7..2^10 beside the paper's Algorithm 1 times, and 2^11, 2^12 with every row formed into a
    reused buffer and Theta~ not kept (PC_ALG1_DISCARD: it would need 0.8-3 TB; rows that keep a
    coarse wavelet reach its whole support); the time against eta at 256^2 for both
    threshold rules (the paper's timing-vs-precision figure); and, when checking, the max error of
    a small case against the oracle's dense Algorithm 1.  Each call is synchronous; wall time
    around it (host planning and the allocation of Theta~ included) and the device time of its
    four stages (CUDA events)."""
    import time
    import torch
    import pc_inputs as P

    peak, _ = _peaks()

    def one(name, n, eta, rule, flags=0):
        rec = {"operator": name, "side": n, "eta": eta, "rule": "hard" if rule else "schur"}
        if flags:
            rec["theta_kept"] = False
        a = None
        try:
            op = P.workload(name, n=n, seed_offset=rank)
            desc = pw.make_desc(2, n, op.levels, op.delta, op.m, op.r, gap=-1, precision=pw.PC_FP32,
                                family=op.family)
            u = torch.tensor(op.u, device=dev)
            v = torch.tensor(op.v, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            a = pw.PCAlg1(desc, u, v, eta, rule=rule, flags=flags)
            wall = time.perf_counter() - t0
            prod_ms = float(a.stage_ms[3])
            gbs = 4.0 * a.nnz / (prod_ms * 1e-3) / 1e9          # FP32 entries written by the products
            rec.update({"N": op.N, "m": op.m, "s": round(wall, 4),
                        "stage_ms": {k: round(float(x), 3) for k, x in
                                     zip(("generators", "thresholds", "synthesis", "products"), a.stage_ms)},
                        "nnz": a.nnz, "entries_per_row": round(a.nnz / op.N, 1),
                        "kept_per_row_per_term": round(float(a.kept.sum()) / op.N / op.m, 1),
                        "products_roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak,
                                              "unit": "GB/s", "frac": round(gbs / peak, 4),
                                              "entries_per_s": round(a.nnz / (prod_ms * 1e-3), -6)}})
        except Exception as e:                       # recorded, not fatal to the bench line
            rec["error"] = str(e)[:160]
        finally:
            if a is not None:
                a.close()
        return rec

    one("op1", 128, 5e-4, 1)                         # first call: module set-up
    out = {"sweep": [], "vs_eta_256": []}
    for name in ops:
        for n in tuple(sides) + tuple(discard_sides):
            rec = one(name, n, eta, 1, pw.PC_ALG1_DISCARD if n in discard_sides else 0)
            rec["paper_alg1_s"] = PAPER_ALG1_S[name][n] if eta == 5e-4 else None
            if "s" in rec and rec["paper_alg1_s"]:
                rec["paper_over_gpu"] = round(rec["paper_alg1_s"] / rec["s"], 1)
            out["sweep"].append(rec)
    for eta in ((1.0, 5e-4, 1e-6, 2e-11) if vs_eta else ()):     # the eta of the paper's figure
        for rule in (0, 1):
            for name in ops:
                out["vs_eta_256"].append(one(name, 256, eta, rule))
    if check:
        import oracle
        errs = {}
        for rule in (0, 1):
            n, m, r = 32, 3, 2
            u = P.normal(P.BASE_SEED + 901, m * (2 * r + 1) ** 2).reshape(m, -1)
            v = P.uniform(P.BASE_SEED + 902, m * n * n).reshape(m, -1) + 0.1
            op = P.Operator("alg1-check", 2, n, 3, 3, r, u, v, gap=-1)
            To, _, _ = oracle.alg1_dense(op, 1e-3, rule=rule)
            for fp32 in (False, True):
                desc = pw.make_desc(2, n, 3, 3, m, r, gap=-1, precision=pw.PC_FP32 if fp32 else pw.PC_FP64)
                a = pw.PCAlg1(desc, u, v, 1e-3, rule=rule)
                T = a.dense()
                a.close()
                errs[f"{'hard' if rule else 'schur'}_{'fp32' if fp32 else 'fp64'}"] = \
                    float(np.abs(T - To).max() / np.abs(To).max())
        out["max_rel_err_vs_oracle_32x32"] = errs
    return out


# ---------------- the oracle leg: CPU baseline and per-result errors against the FP64 oracle ----------------
# Everything below runs outside the timed regions; it is the one part of the GPU arm that calls
# the oracle (test infrastructure), and only to time it and to compare results with it.
def _stratified(op, seed, per_band=1, bands=None):
    """Seeded indices: per_band per band (band b of `bands`, default all), canonical order."""
    rng = np.random.default_rng(seed)
    n, L, d = op.n, op.levels, op.d
    starts = [(0, (n >> L) ** d)]
    for j in range(L, 0, -1):
        nb = (n >> j) ** d
        for t in range(1 if d == 1 else 3):
            starts.append(((n >> j) if d == 1 else nb * (1 + t), nb))
    pick = []
    for b, (off, size) in enumerate(starts):
        if bands is None or b in bands:
            pick += (off + rng.integers(0, size, per_band)).tolist()
    return np.array(sorted(set(pick)), dtype=np.int64)


def oracle_column_error(g, op, cols, nthreads=0):
    """max |Theta - Theta_oracle| / max |Theta_oracle| over the pattern entries of `cols`,
    gathering only those entries from the device."""
    import torch
    import oracle
    T = oracle.theta_columns(op, cols, nthreads=nthreads)
    vals = g.values()
    err = ref = 0.0
    for c, lam in enumerate(cols):
        mus = np.nonzero(oracle.pattern_column(op, int(lam)))[0].astype(np.int64)
        pos = g.lookup(mus, np.full(mus.size, lam, dtype=np.int64))
        if (pos < 0).any():
            return float("inf")
        got = vals[torch.as_tensor(pos, device=vals.device)].double().cpu().numpy()
        err = max(err, float(np.abs(got - T[c][mus]).max(initial=0.0)))
        ref = max(ref, float(np.abs(T[c][mus]).max(initial=0.0)))
    return err / ref if ref else 0.0


def _flipped(op):
    """Mirrored kernels and the other order: column mu of its Theta is row mu of op's
    (Theta_0(u)^T = Theta_1(flip u))."""
    import copy
    o = copy.copy(op)
    o.u = np.ascontiguousarray(op.u[:, ::-1])
    o.order = 1 - op.order
    return o


def oracle_apply_error(op, x, y, rows, nthreads=0):
    """max over right-hand sides of ||y - Theta_oracle x|| / ||Theta_oracle x|| on `rows`."""
    import oracle
    R = oracle.theta_columns(_flipped(op), rows, nthreads=nthreads)
    ref = np.zeros((rows.size, x.shape[1]))
    for i, mu in enumerate(rows):
        mask = oracle.pattern_column(op, int(mu))      # the pattern is symmetric
        ref[i] = R[i][mask] @ x[mask]
    got = y[rows]
    return float((np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)).max())


def oracle_grad_error(pw, g, op, cols, seed, nthreads=0):
    """Seeded N(0,1) dL/dTheta on the pattern entries of `cols`: the GPU's dL/du, dL/dv against
    the oracle's adjoint, element-wise: max |g - g_ref| / max |g_ref| over du and dv."""
    import torch
    import oracle
    import pc_inputs as P
    G = np.zeros((cols.size, op.N))
    Gd = torch.zeros(g.nnz, dtype=g.dtype, device="cuda")
    for c, lam in enumerate(cols):
        mus = np.nonzero(oracle.pattern_column(op, int(lam)))[0].astype(np.int64)
        vals = P.normal(seed + c, mus.size)
        G[c, mus] = vals
        pos = g.lookup(mus, np.full(mus.size, lam, dtype=np.int64))
        Gd[torch.as_tensor(pos, device="cuda")] = torch.tensor(vals, dtype=g.dtype, device="cuda")
    du, dv = g.backward(Gd)
    g.sync()
    du_ref, dv_ref = oracle.theta_grad(op, cols, G, nthreads=nthreads)
    e = [float(np.abs(a.double().cpu().numpy() - b).max() / np.abs(b).max()) for a, b in ((du, du_ref), (dv, dv_ref))]
    del Gd
    return max(e)


def fd_grad_error(pw, nparams=8, seed=3):
    """Differentiation workload (2-D 128^2, db4, L=3, m=9, 11x11 kernels): the GPU's FP32 gradient
    (forward and backward on the device) of L = ||Theta_P(u) - Theta_P(u_target)||^2 over a
    seeded sample of columns, against FP64 central differences (step 1e-6) of the same loss
    evaluated by the oracle, on `nparams` seeded parameters (half kernel taps, half window pixels
    inside a sampled column's support): max per parameter of |g - fd| / max(|fd|, 1e-3 max|g|)."""
    import torch
    import oracle
    import pc_inputs as P
    op = P.workload("c3")
    tgt = P.workload("c3")
    tgt.u = op.extra["u_target"]
    cols = _stratified(op, 9, per_band=3)
    masks = np.array([oracle.pattern_column(op, int(lam)) for lam in cols])
    Tt = oracle.theta_columns(tgt, cols)

    def loss(u, v):
        return float((((oracle.theta_columns(op, cols, u=u, v=v) - Tt) * masks) ** 2).sum())

    mk = lambda o: pw.PCOperator(pw.desc_of(o), torch.tensor(o.u, dtype=torch.float32, device="cuda"),
                                 torch.tensor(o.v, dtype=torch.float32, device="cuda"))
    g, t = mk(op), mk(tgt)
    g.assemble()
    t.assemble()
    mus = np.arange(op.N, dtype=np.int64)
    pos = np.concatenate([g.lookup(mus[m], np.full(int(m.sum()), lam, dtype=np.int64)) for lam, m in zip(cols, masks)])
    pd = torch.as_tensor(pos, device="cuda")
    G = torch.zeros(g.nnz, dtype=torch.float32, device="cuda")
    G[pd] = 2.0 * (g.values()[pd] - t.values()[pd])
    du, dv = g.backward(G)
    g.sync()
    du, dv = du.double().cpu().numpy(), dv.double().cpu().numpy()
    scale = max(np.abs(du).max(), np.abs(dv).max())
    rng = np.random.default_rng(P.BASE_SEED + seed)
    h, worst = 1e-6, 0.0
    for i in range(nparams):
        k = int(rng.integers(op.m))
        u0, v0 = op.u.copy(), op.v.copy()
        if i % 2 == 0:
            tp = int(rng.integers(op.u.shape[1]))
            up, um = u0.copy(), u0.copy()
            up[k, tp] += h
            um[k, tp] -= h
            fd, got = (loss(up, v0) - loss(um, v0)) / (2 * h), du[k, tp]
        else:
            lam = int(cols[int(rng.integers(cols.size))])
            e = np.zeros(op.N)
            e[lam] = 1.0
            supp = np.nonzero(oracle.idwt(op.d, op.n, op.levels, op.delta, e))[0]
            x = int(supp[int(rng.integers(supp.size))])
            vp, vm = v0.copy(), v0.copy()
            vp[k, x] += h
            vm[k, x] -= h
            fd, got = (loss(u0, vp) - loss(u0, vm)) / (2 * h), dv[k, x]
        worst = max(worst, abs(got - fd) / max(abs(fd), 1e-3 * scale))
    g.close()
    t.close()
    return worst, nparams


def _ev(stream, fn, reps=3, flush=None):
    """Median CUDA-event time (ms) of fn() on `stream` over `reps` runs (L2 flushed before each)."""
    import torch
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def run_batch(pw, rank, dev, stream, flush, check):
    """Batched FP32 assembly of the 64 uneven operators (one CUDA graph) against the plain
    FP64 assembly of each operator alone; errors against the oracle on two seeded columns per
    operator (one from the finest band, one from any band)."""
    import torch
    import pc_inputs as P
    bops = P.batch_workload(64, seed_offset=rank)
    bg = [pw.PCOperator(pw.desc_of(o, pw.PC_FP32, 0), torch.tensor(o.u, dtype=torch.float32, device=dev),
                        torch.tensor(o.v, dtype=torch.float32, device=dev)) for o in bops]
    bnnz = sum(x.nnz for x in bg)
    batch = pw.PCBatch(bg)                 # plans the queue, runs once, captures the graph
    for _ in range(2):
        batch.run()
    batch_ms = _ev(stream, batch.run, reps=5, flush=flush)
    for x in bg:
        x.sync()
    items = batch.items
    err = None
    if check and rank == 0:
        err = 0.0
        for i, (o, x) in enumerate(zip(bops, bg)):
            nb = 1 + o.levels * (1 if o.d == 1 else 3)
            cols = np.concatenate([_stratified(o, 40 + i, 1, bands={nb - 1}), _stratified(o, 80 + i, 1)])[:2]
            err = max(err, oracle_column_error(x, o, cols))
    batch.close()
    for x in bg:
        x.close()
    del bg
    # plain FP64: one operator per assembly call, the same kernels instantiated in FP64
    f64 = 0.0
    for o in bops:
        x = pw.PCOperator(pw.desc_of(o, pw.PC_FP64, 0), torch.tensor(o.u, dtype=torch.float64, device=dev),
                          torch.tensor(o.v, dtype=torch.float64, device=dev))
        x.assemble()
        f64 += _ev(stream, x.assemble, reps=1, flush=flush)
        x.close()
    peak, _ = _peaks()
    gbs = 4 * bnnz / (batch_ms * 1e-3) / 1e9
    return {"ops": 64, "nnz": bnnz, "items": items, "fp32_ms": round(batch_ms, 3),
            "entries_per_s": bnnz / (batch_ms * 1e-3), "hbm_gbs_alg": round(gbs, 1), "hbm_frac": round(gbs / peak, 4),
            "fp64_plain_ms": round(f64, 2), "vs_fp64_plain": round(f64 / batch_ms, 2),
            "max_rel_err": err, "tol": 1e-5}


def run_c5(pw, dev, stream, flush, check):
    """The large workload (2-D 1024^2, db4, L=5, m=64, 31x31 Gaussian * motion kernels): FP32
    assembly with its BF16 copy, the BF16 apply to 16 right-hand sides, the backward; errors
    against the oracle on seeded columns / rows of the finest and coarsest bands."""
    import torch
    import pc_inputs as P
    op = P.workload("c5")
    g = pw.PCOperator(pw.desc_of(op, pw.PC_FP32, 1), torch.tensor(op.u, dtype=torch.float32, device=dev),
                      torch.tensor(op.v, dtype=torch.float32, device=dev))
    pw.pc_autotune(g.h)
    nrhs = 16
    xh = P.normal(P.BASE_SEED + 98, op.N * nrhs).reshape(op.N, nrhs)
    x = torch.tensor(xh, dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    K = (2 * op.r + 1) ** 2
    du = torch.empty((op.m, K), dtype=torch.float32, device=dev)
    dv = torch.empty((op.m, op.N), dtype=torch.float32, device=dev)
    g.assemble()
    asm = _ev(stream, g.assemble, flush=flush)
    app = _ev(stream, lambda: pw.pc_apply(g.h, x, y, nrhs), flush=flush)
    th = g.values()
    bwd = _ev(stream, lambda: pw.pc_backward(g.h, th, du, dv), flush=flush)
    g.sync()
    peak, _ = _peaks()
    out = {"nnz": g.nnz, "assemble_ms": round(asm, 2), "entries_per_s": g.nnz / (asm * 1e-3),
           "hbm_frac_alg": round(6 * g.nnz / (asm * 1e-3) / 1e9 / peak, 4),
           "apply16_bf16_ms": round(app, 2), "bwd_ms": round(bwd, 2)}
    if check:
        nb = 1 + 3 * op.levels
        cols = np.concatenate([_stratified(op, 51, 2, bands={nb - 1}), _stratified(op, 52, 1, bands={0})])
        out["asm_err"] = oracle_column_error(g, op, cols)
        pw.pc_apply(g.h, x, y, nrhs)
        torch.cuda.synchronize()
        yh = y.double().cpu().numpy()
        out["apply_err"] = oracle_apply_error(op, xh, yh, _stratified(op, 53, 2))
        out["bwd_err"] = oracle_grad_error(pw, g, op, _stratified(op, 54, 2, bands={nb - 1}), P.BASE_SEED + 700,
                                           nthreads=4)
    g.close()
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2005_09870_gb300 as pw
    import pc_inputs as P

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if args.only_alg1:
        # the thresholded Algorithm 1 leg alone (no throughput line), e.g. to profile it
        sides = tuple(int(x) for x in args.alg1_sides.split(",") if x)
        out = run_alg1(pw, rank, dev, not args.no_check, sides=sides, discard_sides=(),
                       ops=tuple(args.alg1_ops.split(",")), vs_eta=False, eta=args.alg1_eta)
        if rank == 0:
            print(json.dumps({"alg1_thresholded": out}), flush=True)
        return
    stream = torch.cuda.current_stream()
    op = rank_workload(args.workload, rank)
    u = torch.tensor(op.u, dtype=torch.float32, device=dev)
    v = torch.tensor(op.v, dtype=torch.float32, device=dev)
    g = pw.PCOperator(pw.desc_of(op, pw.PC_FP32, 1), u, v)
    if not args.no_tune:
        pw.pc_autotune(g.h)                 # per-band thread-group shapes (untimed setup)
    nnz = g.nnz
    nrhs = 16
    xh = P.normal(P.BASE_SEED + 99 + rank, op.N * nrhs).reshape(op.N, nrhs)
    x = torch.tensor(xh, dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    K = (2 * op.r + 1) ** op.d
    du = torch.empty((op.m, K), dtype=torch.float32, device=dev)
    dv = torch.empty((op.m, op.N), dtype=torch.float32, device=dev)
    theta_vals = g.values()                # dL/dTheta = Theta for L = 1/2 ||Theta||^2
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]

    def step(e=None):
        if e: e[0].record(stream)
        pw.pc_assemble_stage(g.h, 0)
        if e: e[1].record(stream)
        pw.pc_assemble_stage(g.h, 1)
        if e: e[2].record(stream)
        pw.pc_apply(g.h, x, y, nrhs)
        if e: e[3].record(stream)
        pw.pc_backward(g.h, theta_vals, du, dv)
        if e: e[4].record(stream)

    for _ in range(args.warmup):
        step()
    g.sync()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = pw.pc_launch_counter()
    with Clocks(local_rank) as clk:
        for i in range(args.steps):
            flush.zero_()                   # L2 flush between steps (not inside the timed events)
            step(ev[i])
        torch.cuda.synchronize()
    launches = pw.pc_launch_counter() - launches0
    if world > 1:
        torch.distributed.barrier()
    g.sync()
    ph = np.array([[ev[i][k].elapsed_time(ev[i][k + 1]) for k in range(4)] for i in range(args.steps)])
    step_ms = ph.sum(axis=1)
    ms = max_over_ranks(float(step_ms.mean()), dev, world)
    prep_ms, rows_ms, apply_ms, bwd_ms = (float(a) for a in ph.mean(axis=0))
    value = job_value(world, nnz, ms)
    y_step = y.double().cpu().numpy()

    # ---------------- end to end through the C-ABI with host buffers ----------------
    u_h = torch.tensor(op.u, dtype=torch.float32).pin_memory()
    v_h = torch.tensor(op.v, dtype=torch.float32).pin_memory()
    x_h = x.cpu().pin_memory()
    y_h = torch.empty_like(x_h).pin_memory()
    du_h = torch.empty(du.shape, dtype=torch.float32).pin_memory()
    dv_h = torch.empty(dv.shape, dtype=torch.float32).pin_memory()
    h2d = (u_h.numel() + v_h.numel() + x_h.numel()) * 4
    d2h = (y_h.numel() + du_h.numel() + dv_h.numel()) * 4
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    for i in range(args.steps + args.warmup):
        flush.zero_()
        e = e2e_ev[i - args.warmup] if i >= args.warmup else None
        if e: e[0].record(stream)
        pw.pc_set_params(g.h, u_h, v_h)     # H2D from pinned host memory
        x.copy_(x_h, non_blocking=True)
        step()
        y_h.copy_(y, non_blocking=True)
        du_h.copy_(du, non_blocking=True)
        dv_h.copy_(dv, non_blocking=True)
        if e: e[1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in e2e_ev])), dev, world)
    e2e_value = job_value(world, nnz, e2e_ms)

    # ---------------- plain FP64 single-operator baseline (same kernels in FP64) ----------------
    u64 = torch.tensor(op.u, dtype=torch.float64, device=dev)
    v64 = torch.tensor(op.v, dtype=torch.float64, device=dev)
    g64 = pw.PCOperator(pw.desc_of(op, pw.PC_FP64, 0), u64, v64)
    for _ in range(2):
        g64.assemble()
    fp64_asm_ms = _ev(stream, g64.assemble, flush=flush)
    fp32_asm_ms = prep_ms + rows_ms
    check = rank == 0 and not args.no_check
    err = {}
    if check:
        cols = _stratified(op, 3, per_band=1)
        err["assembly_fp32"] = oracle_column_error(g, op, cols)
        err["assembly_fp64"] = oracle_column_error(g64, op, cols)
        err["apply_bf16"] = oracle_apply_error(op, xh, y_step, _stratified(op, 4, per_band=1))
        err["bwd_vs_oracle"] = oracle_grad_error(pw, g, op, _stratified(op, 5, per_band=1, bands={0, 12}),
                                                 P.BASE_SEED + 800)
        fd, npar = fd_grad_error(pw)
        err["grad_vs_fd_c3"] = fd
        err["tol"] = {"assembly_fp32": 1e-5, "assembly_fp64": 1e-12, "apply_bf16": 1e-2, "bwd_vs_oracle": 1e-5,
                      "grad_vs_fd_c3": 1e-4}
        err["how"] = (f"oracle (FP64 Algorithm 2) on seeded columns of every band (assembly), rows of every band "
                      f"(apply, 16 RHS), seeded dL/dTheta on 2 columns (backward, element-wise); FD: {npar} "
                      f"parameters of the 128^2 differentiation workload, oracle loss, step 1e-6")
    g64.close()

    # ---------------- wavelet-domain deblurring (Section 4.3) on the assembled Theta ----------------
    fista = None
    if not args.no_fista:
        fista = run_fista(pw, g, op, rank, dev, stream, args.fista_iters)

    # ---------------- rooflines: stage 1 of the assembly (the metric's kernels) and the backward ----------------
    peak, peak_kind = _peaks()
    alg_bytes = nnz * (4 + 2) + op.m * op.N * 4     # Theta FP32 + BF16 written once, windows read once
    achieved = alg_bytes / (rows_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": profile_traffic(["k_s_tiles", "k_assemble_batch"]), "alg_bytes": alg_bytes,
            "kernel": "stage 1 of the assembly: k_s_tiles (window sums) + k_assemble_batch (localized transforms)",
            "peak_kind": peak_kind}
    # backward: dL/dTheta read once, dL/dv written and the windows read once, dL/du written
    K = (2 * op.r + 1) ** op.d
    bwd_alg = 4 * nnz + 8 * op.m * op.N + 4 * op.m * K
    bwd_gbs = bwd_alg / (bwd_ms * 1e-3) / 1e9
    roof_bwd = {"bound": "hbm", "achieved": bwd_gbs, "peak": peak, "unit": "GB/s", "frac": bwd_gbs / peak,
                "traffic": profile_traffic(["k_backward_queue", "k_bwd_dv4", "k_bwd_dF_wl"]), "alg_bytes": bwd_alg,
                "kernel": "pc_backward: k_backward_queue (adjoint rows) + k_bwd_dv4 (dL/dv) + k_bwd_dF_wl (dL/dF) "
                          "+ the small adjoint of the filtered wavelets", "peak_kind": peak_kind}
    flops = assembly_flops(op) if op.d == 2 else None
    roof_fp32 = None
    if flops:
        tf = flops / (rows_ms * 1e-3) / 1e12
        roof_fp32 = {"bound": "alu", "achieved": tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": tf / FP32_PEAK_TFLOPS, "flops": flops,
                     "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"}
    g.close()
    del flush
    torch.cuda.empty_cache()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # ---------------- batched FP32 vs plain FP64 on 64 uneven operators ----------------
    batch_info = None if args.no_batch else run_batch(pw, rank, dev, stream, flush, check)
    c5 = None if args.no_c5 else run_c5(pw, dev, stream, flush, check)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, cols, threads, wall = cpu_oracle_rate(op, args.cpu_seconds)
        rate1, cols1, _, wall1 = cpu_oracle_rate(op, min(4.0, args.cpu_seconds / 3), seed=6, nthreads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{cols} uniformly drawn columns of the workload, Algorithm 2 in FP64, {wall:.1f} s",
               "single_thread": {"value": rate1, "unit": UNIT,
                                 "sample": f"{cols1} columns on one core, {wall1:.1f} s"},
               "full_theta_s_extrapolated": nnz / rate}

    sweep = None
    if not args.no_sweep:
        sweep = run_sweep(pw, rank, dev, stream)
    alg1 = None
    if not args.no_alg1:
        alg1 = run_alg1(pw, rank, dev, check)

    clocks = clk.summary()
    if rank == 0:
        r4 = lambda z: None if z is None else float(f"{z:.4g}")
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "nnz": nnz,
            "config": bench_config(world),
            # details first; the driver's record keeps the end of the line
            "symmlet6_sweep": sweep,
            "alg1_thresholded": alg1,
            "fista": fista,
            "roofline_fp32": roof_fp32,
            "phases_ms": {"prepare": prep_ms, "assemble_rows": rows_ms, "apply_16rhs": apply_ms, "backward": bwd_ms},
            "roofline": roof,
            "roofline_bwd": roof_bwd,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms},
            "gpu_launches": int(launches),
            "gpu_launches_per_step": launches / args.steps,
            "clocks": clocks,
            # summary of the metric's own numbers, last
            "c5_1024": c5,
            "batch_c4": batch_info,
            "assembly_c2": {"fp32_ms": r4(fp32_asm_ms), "fp64_plain_ms": r4(fp64_asm_ms),
                            "fp32_vs_fp64": r4(fp64_asm_ms / fp32_asm_ms),
                            "entries_per_s": r4(nnz / (fp32_asm_ms * 1e-3)),
                            "stage1_hbm_frac": r4(achieved / peak)},
            "errors_vs_oracle": {k: (r4(v) if isinstance(v, float) else v) for k, v in err.items()},
            "bwd_ms": r4(bwd_ms),
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-fista", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-c5", action="store_true")
    ap.add_argument("--no-alg1", action="store_true")
    ap.add_argument("--only-alg1", action="store_true", help="run only the thresholded Algorithm 1 leg")
    ap.add_argument("--alg1-sides", default="256", help="sides for --only-alg1, comma separated")
    ap.add_argument("--alg1-ops", default="op1,op2", help="operators for --only-alg1")
    ap.add_argument("--alg1-eta", type=float, default=5e-4, help="eta for --only-alg1")
    ap.add_argument("--fista-iters", type=int, default=50)
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
