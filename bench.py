#!/usr/bin/env python
"""Throughput of the T2 Shuffling PICS solve (one GB300 per rank).

One step = one whole reconstruction of the synthetic knee scan: t2sh_plan (maps,
space-time kernel Psi, step, shifts) + t2sh_solve (A^H y, then 100 FISTA iterations of
normal operator + LLR prox over all 320 slices of 256 x 160, C = 12, T = 80, K = 4,
5 %/echo, lambda = 0.005, b = 8) + t2sh_destroy.  Inputs are device resident when the
timed region starts (the `e2e` figure repeats it through host buffers).  The metric is
slice-iterations per second (slices x iterations / seconds) over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank reconstructs its own copy of the scan (slices are independent
problems: weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "slice-iterations/s (T2 Shuffling FISTA PICS solve, full scan)"
UNIT = "slice-iter/s"
KERNEL_FILES = ["t2sh_device.cuh", "t2sh_plan.h", "k_fft.cu", "k_fft_fast.cu", "k_col_tma.cu", "k_col_pr.cu", "k_fused.cu", "k_llr.cu",
                "k_prep.cu", "t2sh_api.cu"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--slices", type=int, default=None, help="fewer slices (profiling runs only)")
    ap.add_argument("--iters", type=int, default=None, help="fewer iterations (profiling runs only)")
    ap.add_argument("--precision", choices=["fp32", "mixed"], default="fp32",
                    help="mixed: column DFTs as split-BF16 GEMMs on the tensor cores (FP32 accumulation)")
    ap.add_argument("--form", choices=["batched", "per-slice"], default="batched",
                    help="per-slice: one plan and one solve per slice (the plain per-slice form)")
    ap.add_argument("--col-variant", type=int, default=None,
                    help="pin the column-pass variant (t2sh_configure); default: the plan's own choice")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solver", choices=["fista", "admm"], default="fista",
                    help="admm: t2sh_solve_admm (CG alpha-updates); an iteration is one outer ADMM iteration")
    ap.add_argument("--rho", type=float, default=0.5)
    ap.add_argument("--cg-iters", type=int, default=3)
    ap.add_argument("--post-te", default="",
                    help="comma-separated echo indices: each step also forms TE images (t2sh_postprocess, pf 0.65)")
    ap.add_argument("--wavelet", type=int, default=0,
                    help="levels of the wavelet soft-threshold (t2sh_wavelet_denoise) each step applies to the "
                         "solved volume; 0: none")
    ap.add_argument("--wavelet-tau", type=float, default=1e-3)
    ap.add_argument("--preproc", action="store_true",
                    help="time the pre-processing instead (coil compression 16 -> C channels and sparse lines -> "
                         "projected k-space for the whole scan); prints its own JSON line")
    ap.add_argument("--workload", choices=["knee", "paper", "batch3"], default="knee",
                    help="paper: the Table I scan (288 slices of 260x240, C=7, M=2, b=12, 250 iterations); "
                         "batch3: three scans of different shapes in one batched solve (t2sh_solve_batch)")
    ap.add_argument("--eig", choices=["fp32", "fp64"], default="fp32",
                    help="precision of the LLR K x K eigendecomposition (fp64: T2SH_EIG_FP64)")
    ap.add_argument("--batch-schedule", choices=["list", "per-scan"], default="list",
                    help="batch3: one LLR launch per iteration over all scans (list) or one per scan")
    ap.add_argument("--prof-steps", type=int, default=2,
                    help="steps of the separate instrumented pass that gives the per-kernel times")
    return ap.parse_args()


def workload(args):
    import t2sh_synth as synth
    if getattr(args, "workload", "knee") == "batch3":
        sh = synth.KNEE_320x256x160
    else:
        sh = synth.PAPER_288x260x240 if getattr(args, "workload", "knee") == "paper" else synth.KNEE_320x256x160
    S = args.slices or sh.nslices
    iters = args.iters if args.iters is not None else sh.iters
    return sh, S, iters


def batch3_config(n):
    import t2sh_synth as synth
    scans = [f"{sh.nslices} x {sh.ny}x{sh.nz} C={sh.ncoils}" for sh in synth.BATCH_SCANS]
    return {"workload": "three synthetic scans in one batched solve (t2sh_solve_batch): " + "; ".join(scans) +
                        "; T=80, K=4, M=1, 5%/echo, b=8, lambda=0.005, 100 FISTA iterations each",
            "scans": scans, "slices": sum(sh.nslices for sh in synth.BATCH_SCANS), "iterations": 100,
            "parallelism": f"scans x slices, dp{n}",
            "l2": "inputs larger than L2 (per-iteration working set > 20 GB)"}


def config_dict(sh, S, iters, n):
    kind = "paper-shape (Table I)" if sh.nmaps > 1 else "knee"
    return {"workload": f"synthetic {kind} scan, {S} slices of {sh.ny}x{sh.nz}, C={sh.ncoils}, T={sh.nechoes}, "
                        f"K={sh.nbasis}, M={sh.nmaps}, {sh.frac * 100:.3g}%/echo, b={sh.block}, lambda={sh.lam}, "
                        f"{iters} FISTA iterations",
            "slices": S, "ny": sh.ny, "nz": sh.nz, "coils": sh.ncoils, "echoes": sh.nechoes, "basis": sh.nbasis,
            "maps": sh.nmaps,
            "iterations": iters, "block": sh.block, "lambda": sh.lam, "parallelism": f"slices, dp{n}",
            "l2": "inputs larger than L2 (per-iteration working set > 6 GB)"}


# ------------------------------------------------------------------------------------
# CPU legs: the FP64 oracle on a bounded sample of the workload
# ------------------------------------------------------------------------------------
CPU_SAMPLE_SLICES = 8


def sample_slices(sh, n=CPU_SAMPLE_SLICES):
    """A seeded choice of n distinct slices of the scan (sorted)."""
    import numpy as np
    import t2sh_synth as synth
    rng = synth.rng_for(sh.seed, 7)
    return sorted(int(s) for s in rng.choice(sh.nslices, size=min(n, sh.nslices), replace=False))


def shape_by_name(name):
    import t2sh_synth as synth
    return getattr(synth, name)


def shape_name(sh):
    import t2sh_synth as synth
    for n in ("KNEE_320x256x160", "PAPER_288x260x240", "SINGLE_SLICE_64x48"):
        if getattr(synth, n) is sh:
            return n
    raise ValueError(sh.name)


def write_sample(sh, path):
    """The oracle's own acquisition of the sample slices (projected k-space, float64
    structure rounded to the float32 / complex64 values a GPU receives), saved to path."""
    import numpy as np
    from oracle.acquire import proj_scan
    sl = sample_slices(sh)
    phi, mask, maps, ytil = proj_scan(sh, sl)
    np.savez(path, slices=np.array(sl), phi=phi.astype(np.float32), mask=mask, maps=maps.astype(np.complex64),
             ytil=ytil.astype(np.complex64))


_W = {}


def _worker_init(path, name):
    import numpy as np
    d = np.load(path)
    _W.update({k: d[k] for k in d.files})
    _W["sh"] = shape_by_name(name)


def _worker_fista(i, iters):
    """One sample slice through the oracle's FISTA; returns (wall start, wall end, alpha)."""
    import oracle as O
    sh = _W["sh"]
    phi = _W["phi"].astype("float64")
    maps = _W["maps"][i].astype("complex128")
    y = _W["ytil"][i].astype("complex128")
    t0 = time.time()
    x = O.fista(y, "proj", maps, _W["mask"], phi, sh.lam, sh.block, iters, sh.seed)
    return t0, time.time(), x


def oracle_pool(path, name, nproc):
    import multiprocessing as mp
    env = {"OPENBLAS_NUM_THREADS": "1", "OMP_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
    os.environ.update(env)
    return mp.get_context("spawn").Pool(nproc, initializer=_worker_init, initargs=(path, name))


def oracle_round(pool, n, iters):
    """All n sample slices at once, one process each; wall seconds from the first start
    to the last end, and the results."""
    res = pool.starmap(_worker_fista, [(i, iters) for i in range(n)])
    return max(r[1] for r in res) - min(r[0] for r in res), [r[2] for r in res]


def cpu_baseline_main(name, path, iters):
    """Child process of cpu_baseline(): sample inputs, then the oracle on every sample
    slice at once; writes the oracle's results next to the inputs, prints a JSON line."""
    import numpy as np
    sh = shape_by_name(name)
    write_sample(sh, path)
    n = len(sample_slices(sh))
    with oracle_pool(path, name, n) as pool:
        wall, xs = oracle_round(pool, n, iters)
    np.save(path + ".alpha.npy", np.stack(xs))
    print(json.dumps({"wall_s": wall, "slices": n, "iters": iters}))


def cpu_baseline(sh, gpu_solve=None):
    """The FP64 oracle on the seeded 8-slice sample x the workload's iterations, one
    process per slice on the host cores (one BLAS thread each), in a child process.  With
    gpu_solve, the same inputs are also solved on the GPU and compared slice by slice."""
    import tempfile
    import numpy as np
    name = shape_name(sh)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "sample.npz")
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = "import sys; sys.path.insert(0, %r); import bench; bench.cpu_baseline_main(%r, %r, %d)" % (
            ROOT, name, path, sh.iters)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1500)
        if r.returncode != 0:
            return {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "error": r.stderr[-400:]}
        info = json.loads(r.stdout.strip().splitlines()[-1])
        n, it, wall = info["slices"], info["iters"], info["wall_s"]
        out = {"value": n * it / wall, "unit": UNIT, "cores": n, "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} seeded slices {sample_slices(sh)} of {sh.nslices} x {it} FISTA iterations, FP64 "
                         f"numpy oracle, one process per slice (1 BLAS thread each), {wall:.1f} s wall",
               "full_scan_s_extrapolated": sh.nslices * it / (n * it / wall),
               "extrapolation": f"x{sh.nslices / n:g} slices at the measured rate (not measured)"}
        if gpu_solve is not None:
            d = np.load(path)
            ref = np.load(path + ".alpha.npy")
            got = gpu_solve(d["phi"], d["mask"], d["maps"], d["ytil"]).astype(np.complex128)
            e = [float(np.linalg.norm(got[i] - ref[i]) / np.linalg.norm(ref[i])) for i in range(n)]
            out["nrmse_vs_oracle"] = {"max": max(e), "per_slice": e}
    return out


def run_reference(args):
    """The oracle as it stands, on the same 8-slice sample as cpu_baseline, one process per
    slice; each step is every sample slice through REF_ITERS FISTA iterations."""
    import tempfile
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sh, S, iters = workload(args)
    if sh is None:
        sh = shape_by_name("KNEE_320x256x160")
    per_step = 10
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "sample.npz")
        write_sample(sh, path)
        n = len(sample_slices(sh))
        with oracle_pool(path, shape_name(sh), n) as pool:
            for _ in range(args.warmup):
                oracle_round(pool, n, per_step)
            tot = 0.0
            for _ in range(args.steps):
                tot += oracle_round(pool, n, per_step)[0]
    v = n * per_step * args.steps / tot
    cfg = config_dict(sh, S, iters, args.gpus) if args.workload != "batch3" else batch3_config(args.gpus)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": n, "host_cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"each step: {n} seeded slices {sample_slices(sh)} x {per_step} FISTA "
                                       f"iterations, FP64 numpy oracle, one process per slice (1 BLAS thread "
                                       f"each)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------
# GPU leg
# ------------------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        rows = []
        for ln in (self.out or "").splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        pmax = max(r[2] for r in rows)
        load = [r for r in rows if r[2] >= 0.5 * pmax] or rows
        sm = sorted(r[0] for r in load)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(load), "power_w_max": pmax}


def algorithmic_bytes(S, C, M, K, N):
    """Bytes one launch of each kernel class must move (complex64 = 8 B)."""
    vec = S * M * K * N * 8
    t = S * C * K * N * 8
    maps = S * C * M * N * 8
    return {"row_fwd": vec + maps + t, "row_adj": t + maps + vec, "col": 2 * t, "llr": 6 * vec,
            "band": 2 * t + maps + 5 * vec}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_sha1():
    h = hashlib.sha1()
    for f in KERNEL_FILES:
        with open(os.path.join(ROOT, "paper_1809_04195_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(kernel):
    """DRAM bytes per full-size launch from the committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    e = t.get(kernel)
    if not e or e.get("source_sha1") != kernel_source_sha1():
        return None
    return e.get("dram_bytes_per_launch")


def pipelined_steps(make, solve, n):
    """Run n steps where step i solves the plan from make(i) while make(i + 1) runs on a
    second host thread.  make(i) returns (plan, seconds spent making it); every plan is
    closed after its solve.  Returns the summed seconds per phase: plan (on the second
    thread, overlapped), wait (for a plan to be ready), solve, destroy."""
    from concurrent.futures import ThreadPoolExecutor
    t = {"plan": 0.0, "wait": 0.0, "solve": 0.0, "destroy": 0.0}
    with ThreadPoolExecutor(max_workers=1) as ex:
        fut = ex.submit(make, 0) if n > 0 else None
        for i in range(n):
            t0 = time.perf_counter()
            p, tp = fut.result()
            t1 = time.perf_counter()
            if i + 1 < n:
                fut = ex.submit(make, i + 1)
            try:
                solve(p)
                t2 = time.perf_counter()
            finally:
                p.close()
            t3 = time.perf_counter()
            t["plan"] += tp
            t["wait"] += t1 - t0
            t["solve"] += t2 - t1
            t["destroy"] += t3 - t2
    return t


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1809_04195_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_1809_04195_gb300 import t2sh
    from paper_1809_04195_gb300.dist import max_over_ranks, sum_over_ranks

    sh, S, iters = workload(args)
    from paper_1809_04195_gb300.workload import make_scan
    phi_d, mask_d, maps_d, ytil_d = make_scan(sh, S, dev)
    out_d = torch.empty((S, sh.nmaps, sh.nbasis, sh.ny, sh.nz), dtype=torch.complex64, device=dev)
    prec = t2sh.MIXED_BF16 if args.precision == "mixed" else t2sh.FP32
    eflags = t2sh.EIG_FP64 if args.eig == "fp64" else 0
    dims = t2sh.make_dims(sh.ny, sh.nz, sh.ncoils, sh.nechoes, sh.nbasis, nslices=S, nmaps=sh.nmaps, block=sh.block,
                          lam=sh.lam, iters=iters, seed=sh.seed, precision=prec, flags=eflags)
    N = sh.ny * sh.nz
    units = S * iters

    dims1 = t2sh.make_dims(sh.ny, sh.nz, sh.ncoils, sh.nechoes, sh.nbasis, nslices=1, nmaps=sh.nmaps, block=sh.block,
                           lam=sh.lam, iters=iters, seed=sh.seed, precision=prec, flags=eflags)

    post_te = [int(t) for t in args.post_te.split(",") if t.strip()]
    img_d = (torch.empty((S, len(post_te), sh.ny, sh.nz), dtype=torch.float32, device=dev) if post_te else None)

    def step(timing):
        if args.form == "per-slice":  # every slice its own plan and solve, one after the other
            tm = {}
            for s_ in range(S):
                p = t2sh.Plan(dims1, phi_d, mask_d, maps_d[s_:s_ + 1])
                if timing:
                    p.timing(True)
                p.solve(ytil_d[s_:s_ + 1], t2sh.KSPACE_PROJ, out=out_d[s_:s_ + 1])
                for k, (n, m) in p.timing_read().items():
                    a = tm.setdefault(k, [0, 0.0])
                    a[0] += n
                    a[1] += m
                p.close()
            return {k: tuple(v) for k, v in tm.items()}
        p = t2sh.Plan(dims, phi_d, mask_d, maps_d)
        if args.col_variant is not None:
            p.configure(args.col_variant)
        if timing:
            p.timing(True)
        if args.solver == "admm":
            p.solve_admm(ytil_d, t2sh.KSPACE_PROJ, rho=args.rho, cg_iters=args.cg_iters, out=out_d)
        else:
            p.solve(ytil_d, t2sh.KSPACE_PROJ, out=out_d)
        if args.wavelet:
            p.wavelet_denoise(out_d, args.wavelet_tau, args.wavelet)
        if post_te:
            p.postprocess(out_d, post_te, pf=0.65, out=img_d)
        tm = p.timing_read()  # launch counts always; per-class milliseconds only when timing
        p.close()
        return tm

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # timed region: no per-kernel instrumentation on the stream
    launched = 0
    with Clocks(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(args.steps):
            launched += sum(n for n, _ in step(False).values())
        t1.record()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(t0.elapsed_time(t1))
    value = sum_over_ranks(units * args.steps) / (ms / 1000.0)
    # per-kernel times: a separate pass of the same steps with every launch of the plan
    # bracketed by CUDA events on its stream
    totals = {}
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    prof_steps = max(1, args.prof_steps)
    pe0.record()
    for _ in range(prof_steps):
        for k, (n, m) in step(True).items():
            a = totals.setdefault(k, [0, 0.0])
            a[0] += n
            a[1] += m
    pe1.record()
    torch.cuda.synchronize()
    prof_ms = pe0.elapsed_time(pe1) / prof_steps

    # e2e: the same reconstruction through host buffers (pinned), copies inside the timing
    e2e = None
    if not args.no_e2e:
        import numpy as np
        hphi = phi_d.cpu().numpy()
        hmask = mask_d.cpu().numpy()
        hmaps = maps_d.cpu().pin_memory()
        hy = ytil_d.cpu().pin_memory()
        hout = torch.empty(out_d.shape, dtype=torch.complex64).pin_memory()
        hd = t2sh.make_dims(sh.ny, sh.nz, sh.ncoils, sh.nechoes, sh.nbasis, nslices=S, nmaps=sh.nmaps, block=sh.block,
                            lam=sh.lam, iters=iters, seed=sh.seed, precision=prec, flags=t2sh.HOST_IO | eflags)

        phases = [0.0, 0.0, 0.0]  # plan, solve (host buffers in and out), destroy

        def hsolve(p):
            if args.solver == "admm":
                p.solve_admm(hy, t2sh.KSPACE_PROJ, rho=args.rho, cg_iters=args.cg_iters, out=hout)
            else:
                p.solve(hy, t2sh.KSPACE_PROJ, out=hout)

        def hstep():
            t0 = time.perf_counter()
            p = t2sh.Plan(hd, hphi, hmask, hmaps)
            t1 = time.perf_counter()
            hsolve(p)
            t2 = time.perf_counter()
            p.close()
            t3 = time.perf_counter()
            phases[0] += t1 - t0
            phases[1] += t2 - t1
            phases[2] += t3 - t2

        hstep()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        phases[:] = [0.0, 0.0, 0.0]
        e0 = time.perf_counter()
        for _ in range(args.steps):
            hstep()
        torch.cuda.synchronize()
        es_seq = max_over_ranks(time.perf_counter() - e0)
        seq = {"value": sum_over_ranks(units * args.steps) / es_seq, "full_scan_s": es_seq / args.steps,
               "ms_per_step": {"plan": 1000 * phases[0] / args.steps, "solve": 1000 * phases[1] / args.steps,
                               "destroy": 1000 * phases[2] / args.steps}}

        # pipelined: scan i+1's plan (maps, basis and mask copied from the host, Psi, step) is
        # made on a second host thread and stream while scan i is solved; every scan's host
        # copies still fall inside the timed region
        streams = (torch.cuda.Stream(), torch.cuda.Stream())
        pp = {"plan": 0.0, "wait": 0.0, "solve": 0.0, "destroy": 0.0}

        def make(i):
            torch.cuda.set_device(local)
            t0 = time.perf_counter()
            p = t2sh.Plan(hd, hphi, hmask, hmaps, stream=streams[i % 2])
            return p, time.perf_counter() - t0

        def pipelined(n):
            for k, v in pipelined_steps(make, hsolve, n).items():
                pp[k] += v

        pipelined(2)  # warm the second stream and thread
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        for k in pp:
            pp[k] = 0.0
        e0 = time.perf_counter()
        pipelined(args.steps)
        torch.cuda.synchronize()
        es = max_over_ranks(time.perf_counter() - e0)
        h2d = hphi.nbytes + hmask.nbytes + hmaps.numel() * 8 + hy.numel() * 8
        e2e = {"value": sum_over_ranks(units * args.steps) / es, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(hout.numel() * 8), "full_scan_s": es / args.steps,
               "api": "t2sh_plan + t2sh_solve with T2SH_HOST_IO (pinned host buffers); the next scan's "
                      "t2sh_plan on a second host thread and stream while the current scan is solved",
               "ms_per_step": {"plan_overlapped": 1000 * pp["plan"] / args.steps,
                               "plan_wait": 1000 * pp["wait"] / args.steps,
                               "solve": 1000 * pp["solve"] / args.steps,
                               "destroy": 1000 * pp["destroy"] / args.steps},
               "sequential": seq}
        del hmaps, hy, hout

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peaks, src = measured_peaks()
    ab = algorithmic_bytes(1 if args.form == "per-slice" else S, sh.ncoils, sh.nmaps, sh.nbasis, N)
    if post_te:  # per echo: alpha and the maps read once, the float image written
        Sx = 1 if args.form == "per-slice" else S
        ab["post"] = len(post_te) * (Sx * sh.nmaps * (sh.nbasis + sh.ncoils) * N * 8 + Sx * N * 4)
    if args.wavelet:  # read + write of each level's lattice, forward and inverse
        L = args.wavelet
        vol = S * sh.nmaps * sh.nbasis * N * 8
        ab["post"] = ab.get("post", 0) + 2 * vol * (8.0 ** -(L - 1) + 2 * sum(8.0 ** -(l - 1) for l in range(1, L)))
    if args.solver == "admm":
        vec = (1 if args.form == "per-slice" else S) * sh.nmaps * sh.nbasis * N * 8
        ab["llr"] = 4 * vec  # read alpha, u; write v, u
        # per outer iteration: init (5 reads, 2 writes) + cg_iters x (dot 2, step 4 + 2, dir 2 + 1);
        # the "cg" timing class counts the init and each CG iteration's three kernels as one unit
        ab["cg"] = (7 + 11 * args.cg_iters) * vec / (1 + args.cg_iters)
    kern = {k: {"launches": n // prof_steps, "ms_total": m / prof_steps, "ms_per_launch": (m / n if n else None),
                "algorithmic_bytes_per_launch": ab.get(k)} for k, (n, m) in totals.items() if n}
    dom = max((k for k in kern if k in ab), key=lambda k: kern[k]["ms_total"])
    avg_s = kern[dom]["ms_per_launch"] / 1000.0
    achieved = ab[dom] / avg_s / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "peak_source": src, "traffic": ncu_traffic(dom),
            "algorithmic_bytes_per_launch": ab[dom],
            "timing": f"per-kernel CUDA events on the plan's stream in a separate instrumented pass of {prof_steps} "
                      f"step(s) after the timed region ({prof_ms:.1f} ms/step instrumented vs "
                      f"{ms / args.steps:.1f} ms/step in the uninstrumented timed region)",
            "per_kernel": {k: {**v, "achieved_gbs": (ab[k] / (v["ms_per_launch"] / 1000.0) / 1e9
                                                     if k in ab and v["ms_per_launch"] else None)}
                           for k, v in kern.items()}}
    plans = S if args.form == "per-slice" else 1
    launches = launched + 2 * plans * args.steps  # + maps/Psi kernels of t2sh_plan
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "full_scan_s": ms / args.steps / 1000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == t2sh.FP32 else "f32 + bf16x3 (column DFTs on tensor cores, f32 accumulate)",
            "data": "synthetic (seeded 3D ellipsoid knee phantom, smooth coil maps, variable-density masks)",
            "config": {**config_dict(sh, S, iters, world), "precision": args.precision, "form": args.form,
                       **({"solver": f"admm rho={args.rho} cg_iters={args.cg_iters}"} if args.solver == "admm" else {}),
                       **({"post_te": post_te} if post_te else {}), "eig": args.eig,
                       **({"wavelet": {"levels": args.wavelet, "tau": args.wavelet_tau}} if args.wavelet else {}),
                       **({"col_variant": args.col_variant} if args.col_variant is not None else {})}, "roofline": roof, "gpu_launches": launches,
            "clocks": clk.summary(), "e2e": e2e}
    if world == 1 and not args.no_cpu_baseline and args.solver == "fista" and args.form == "batched":
        def gpu_solve(phi, mask, maps, ytil):
            import numpy as np
            n = maps.shape[0]
            d = t2sh.make_dims(sh.ny, sh.nz, sh.ncoils, sh.nechoes, sh.nbasis, nslices=n, nmaps=sh.nmaps,
                               block=sh.block, lam=sh.lam, iters=sh.iters, seed=sh.seed, precision=prec, flags=eflags)
            with t2sh.Plan(d, torch.from_numpy(phi).to(dev), torch.from_numpy(mask).to(dev),
                           torch.from_numpy(maps).to(dev)) as p:
                return p.solve(torch.from_numpy(ytil).to(dev), t2sh.KSPACE_PROJ).cpu().numpy()
        line["cpu_baseline"] = cpu_baseline(sh, gpu_solve if S == sh.nslices and iters == sh.iters else None)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batch3(args):
    """Three scans of different shapes (320 x 256x160 C=12, 288 x 240x128 C=8, 256 x 192x192
    C=16; 100 iterations each) reconstructed together by t2sh_solve_batch: one step = the
    plans of all three, the batched solve, the plans destroyed.  Inputs device resident."""
    import torch
    import t2sh_synth as synth
    from paper_1809_04195_gb300 import build as B
    B.build()
    from paper_1809_04195_gb300 import t2sh
    from paper_1809_04195_gb300.workload import make_scan
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    prec = t2sh.MIXED_BF16 if args.precision == "mixed" else t2sh.FP32
    eflags = t2sh.EIG_FP64 if args.eig == "fp64" else 0
    t2sh.batch_schedule(args.batch_schedule == "per-scan")
    scans = []
    for sh in synth.BATCH_SCANS:
        S = args.slices or sh.nslices
        it = args.iters if args.iters is not None else sh.iters
        phi_d, mask_d, maps_d, ytil_d = make_scan(sh, S, dev)
        d = t2sh.make_dims(sh.ny, sh.nz, sh.ncoils, sh.nechoes, sh.nbasis, nslices=S, nmaps=sh.nmaps,
                           block=sh.block, lam=sh.lam, iters=it, seed=sh.seed, precision=prec, flags=eflags)
        out = torch.empty((S, sh.nmaps, sh.nbasis, sh.ny, sh.nz), dtype=torch.complex64, device=dev)
        scans.append((sh, S, it, d, phi_d, mask_d, maps_d, ytil_d, out))
    units = sum(S * it for _, S, it, *_ in scans)

    def step():
        plans = [t2sh.Plan(d, phi, mask, maps) for _, _, _, d, phi, mask, maps, _, _ in scans]
        t2sh.solve_batch(plans, [sc[7] for sc in scans], outs=[sc[8] for sc in scans])
        n = 0
        for p in plans:
            n += sum(k for k, _ in p.timing_read().values()) + 2  # + maps/Psi kernels of t2sh_plan
            p.close()
        return n

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    with Clocks(0) as clk:
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        launched = 0
        for _ in range(args.steps):
            launched += step()
        t1.record()
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    # whole-step roofline: every kernel's algorithmic bytes over the step time (the batched
    # graph overlaps the scans' kernels, so per-kernel event times would not mean much)
    tot = 0
    per_scan = []
    for sh, S, it, *_ in scans:
        ab = algorithmic_bytes(S, sh.ncoils, sh.nmaps, sh.nbasis, sh.ny * sh.nz)
        b = (it - 1) * (ab["row_fwd"] + ab["col"] + ab["row_adj"]) + it * ab["llr"] + ab["col"] // 2 + ab["row_adj"]
        tot += b
        per_scan.append({"scan": f"{S} x {sh.ny}x{sh.nz} C={sh.ncoils}", "iterations": it,
                         "algorithmic_bytes": b})
    peaks, src = measured_peaks()
    achieved = tot / (ms / args.steps / 1000.0) / 1e9
    line = {"metric": METRIC, "value": units * args.steps / (ms / 1000.0), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "full_batch_s": ms / args.steps / 1000.0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if prec == t2sh.FP32 else "f32 + bf16x3 (column DFTs on tensor cores, f32 accumulate)",
            "data": "synthetic (seeded 3D ellipsoid phantoms, smooth coil maps, variable-density masks)",
            "config": {**batch3_config(1), "precision": args.precision, "eig": args.eig,
                       "batch_schedule": args.batch_schedule},
            "roofline": {"bound": "hbm", "kernel": "whole batched solve (all kernels, plans included)",
                         "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "peak_source": src, "traffic": None,
                         "algorithmic_bytes_per_step": tot, "per_scan": per_scan},
            "gpu_launches": launched, "clocks": clk.summary(), "e2e": None,
            "e2e_note": "t2sh_solve_batch takes device buffers only; the host-buffer figure is the knee-scan line's"}
    print(json.dumps(line), flush=True)


def run_preproc(args):
    """Seconds per scan of t2sh_coil_compression + t2sh_preprocess on a synthetic sparse
    acquisition of the workload: the scan's per-echo masks, one fully sampled readout line
    of nx = slices samples for every (t, ky, kz) sampled, 16 receive channels compressed
    to the scan's C virtual channels (24^3 calibration window), random line data."""
    import numpy as np
    import torch
    import t2sh_synth as synth
    from paper_1809_04195_gb300 import build as B
    B.build()
    from paper_1809_04195_gb300 import t2sh
    sh, S, _ = workload(args)
    dev = torch.device("cuda", 0)
    phi, mask, _ = synth.scan_common(sh)
    t, a, b = (v.astype(np.int32) for v in np.nonzero(mask))
    nchan, nx = 16, S
    gen = torch.Generator(device=dev)
    gen.manual_seed(sh.seed)
    lines = torch.randn((len(t), nchan, nx), dtype=torch.complex64, device=dev, generator=gen)
    phi_d = torch.from_numpy(phi.astype(np.float32)).to(dev)

    def step():
        w = t2sh.coil_compression(lines, t, a, b, sh.ny, sh.nz, sh.nechoes, window=24, ncomp=sh.ncoils)
        return t2sh.preprocess(lines, t, a, b, w, phi_d, sh.ny, sh.nz)

    for _ in range(args.warmup):
        out = step()
    del out
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        out = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    in_bytes = lines.numel() * 8
    out_bytes = out[0].numel() * 8 + out[1].numel()
    print(json.dumps({"metric": "pre-processing seconds per scan (coil compression + sparse lines to projected "
                                "k-space)", "value": ms / 1000.0, "unit": "s", "higher_is_better": False,
                      "steps": args.steps, "warmup": args.warmup, "n_gpus": 1, "dtype": "f32",
                      "data": "synthetic (random line data at the scan's sampling pattern)",
                      "config": {"workload": config_dict(sh, S, sh.iters, 1)["workload"], "lines": int(len(t)),
                                 "channels": nchan, "virtual_channels": sh.ncoils, "nx": nx,
                                 "line_bytes": int(in_bytes), "projected_bytes": int(out_bytes)},
                      "achieved_gbs_in_plus_out": (in_bytes + out_bytes) / (ms / 1000.0) / 1e9}), flush=True)


def main():
    args = parse()
    if args.preproc:
        run_preproc(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch3":
        run_batch3(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
