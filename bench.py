"""Benchmark of the chi^2 forward-modelling path on the joint multi-band,
multi-epoch fit: 4 bands x 3 epochs of 2048 x 2048 images (each rotated and
dithered, its own 31 x 31 Moffat PSF), 300 Sersic galaxies sharing their
shape across the images with a flux per band, 1000 point sources, a plane sky
per image: 50.3 Mpx and 9036 parameters, the largest configuration that fits
one GPU.

A step is one Levenberg-Marquardt iteration: chi^2 + adjoint gradient at
theta, the Jacobian / J^T W J build, the damped float64 solve, chi^2 at the
trial point and the on-device accept -- every step of the path.  The line also
reports chi^2 + gradient evaluations per second and both numbers for the plain
float64 GPU form on the same GPU, the other workloads under extra_workloads,
and the measured throughput of the arithmetic pipes the rooflines divide by.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload and prints the same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "χ²+gradient evals/s and LM iters/s vs plain FP64 GPU form at stated rel. error"
UNIT = "LM iters/s"
WORKLOAD = "joint_12x2k"
SAMPLE_IMAGES = (0, 4)     # oracle sample: two images of different bands and epochs ...
SAMPLE_SIDE = 256          # ... cut to their central SAMPLE_SIDE x SAMPLE_SIDE pixels
FIT_LEN = 20               # timed LM iterations restart the fit from the initial guess every FIT_LEN steps
F64_LM_STEPS = 3           # float64-form LM iterations timed (each takes seconds on this workload)


def eval_cycle(ctx, theta0, out, n_points=8):
    """chi^2 + gradient evaluations at n_points distinct parameter vectors in
    turn (theta0 scaled by 1 + k 1e-9): every evaluation is at parameters the
    library has not just seen, so nothing cached by parameter value (the
    Sersic b_n memo holds two points) is reused."""
    pts = [theta0 * (1.0 + 1e-9 * (k + 1)) for k in range(n_points)]
    st = {"k": 0}

    def step():
        ctx.eval(pts[st["k"] % n_points], out=out)
        st["k"] += 1
    return step


def rank_max_totals(ms_lists, device, dist=None):
    """Each list of per-step milliseconds summed on this rank, then the
    maximum over ranks: a job of replicas takes as long as its slowest rank."""
    import torch
    tot = torch.tensor([float(sum(m)) for m in ms_lists], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    return [float(x) for x in tot]


def job_rate(world, steps, total_ms):
    """Whole-job rate: every rank ran `steps` units, the job took total_ms."""
    return world * steps / (total_ms / 1e3)


def lm_fit(ctx, theta0, lam0=1e-3):
    """A step function over LM iterations of fits from theta0: every FIT_LEN
    calls it starts a new fit (theta0, lambda0) with lm_iterate, the other
    calls continue it with lm_continue, so that the timed iterations are
    those of fits, not of a fit long converged; .restart() aligns the next
    call with the start of a fit."""
    import torch
    st = {"n": 0}

    def step():
        if st["n"] % FIT_LEN == 0:
            st["theta"] = theta0.clone()
            st["lam"] = torch.full((ctx.n_groups,), lam0, dtype=torch.float64, device=theta0.device)
            st["theta"], st["lam"], _, _ = ctx.lm_iterate(st["theta"], st["lam"], 1)
        else:
            st["theta"], st["lam"], _, _ = ctx.lm_continue(1)
        st["n"] += 1

    step.restart = lambda: st.update(n=0)
    step.state = st
    return step


def workload_config():
    return {"workload": "joint_12x2k: 4 bands x 3 epochs of 2048x2048 FP32 images, each rotated by a random angle and "
                        "dithered by a sub-pixel offset, own 31x31 Moffat PSF (FWHM 2.5-4 px); 300 Sersic (shape shared "
                        "across images, flux per band) + 1000 point sources (position shared, flux per band), plane "
                        "sky per image; 3x3 Gauss-Legendre per pixel; var = model + 1; 9036 parameters",
            "step": "one LM iteration (chi2+adjoint gradient, J^T W J, damped FP64 solve, trial chi2, accept)",
            "fits": f"timed iterations form fits of {FIT_LEN} LM iterations, each from the initial guess (lambda 1e-3)"}


# ---------------------------------------------------------------------------
# problem set-up (inputs only)
# ---------------------------------------------------------------------------

def make_problem():
    from synthetic import configs
    return configs.joint()


def crop_problem(pr, image_ids, r0, c0, H, W):
    """The workload on rows r0..r0+H, columns c0..c0+W of the given images:
    origins moved to the crop's corner, PSFs, masks and noise cut to it, the
    sources whose windows meet it (windows clipped), parameters renumbered
    with shared indices kept shared; one group."""
    import numpy as np
    from synthetic.problem import ImageSpec, Problem, SourceSpec
    imap, images, noise, floors = {}, [], [], []
    for i in image_ids:
        im = pr.images[i]
        A = np.asarray(im.A, float)
        o = np.asarray(im.origin, float) + A @ np.array([c0, r0], float)
        m = None if im.mask is None else im.mask[r0:r0 + H, c0:c0 + W].copy()
        imap[i] = len(images)
        images.append(ImageSpec(H=H, W=W, A=A, origin=o, psf=im.psf, mask=m, group=0))
        noise.append(pr.noise[i][r0:r0 + H, c0:c0 + W].copy())
        floors.append(pr.var_floor[i])
    pmap, srcs = {}, []
    for s in pr.sources:
        if s.image not in imap:
            continue
        x0, x1, y0, y1 = s.win
        x0, x1, y0, y1 = max(x0 - c0, 0), min(x1 - c0, W), max(y0 - r0, 0), min(y1 - r0, H)
        if x0 >= x1 or y0 >= y1:
            continue
        pidx = s.pidx.copy()
        for k in range(8):
            if pidx[k] >= 0:
                pidx[k] = pmap.setdefault(int(pidx[k]), len(pmap))
        srcs.append(SourceSpec(s.type, imap[s.image], (x0, x1, y0, y1), s.psf_convolve, pidx, s.pfix.copy()))
    order = sorted(pmap, key=pmap.get)
    return Problem(pr.name + f"_crop{H}x{W}", images, srcs, len(order), pr.theta_true[order], pr.theta_init[order],
                   quad_order=pr.quad_order, noise=noise, var_floor=floors)


def sample_problem(pr, side):
    """The oracle's sample: the central side x side pixels of two images."""
    H = pr.images[SAMPLE_IMAGES[0]].H
    r0 = (H - side) // 2
    return crop_problem(pr, SAMPLE_IMAGES, r0, r0, side, side)


def jacobian_work(pr):
    """Sum over sources of (Jacobian support pixels x free slots): the size of
    the oracle's per-source render, Jacobian and convolution work, used to
    scale its sample to the whole workload."""
    tot = 0
    for s in pr.sources:
        im = pr.images[s.image]
        h = (im.psf.shape[0] - 1) // 2 if (im.psf is not None and s.psf_convolve) else 0
        tot += _support(s, im, h)[1] * max(1, sum(1 for k in range(8) if s.pidx[k] >= 0))
    return tot


# ---------------------------------------------------------------------------
# CPU oracle leg (runs in a fresh single-threaded interpreter)
# ---------------------------------------------------------------------------

def oracle_worker(n_iter: int, side: int = SAMPLE_SIDE):
    """Time the oracle, as it stands, on the sample crop: n_iter LM iterations."""
    from oracle import astrophot_oracle as O
    from synthetic.problem import attach_data
    import numpy as np
    full = make_problem()
    pr = sample_problem(full, side)
    attach_data(pr, O.model_images(pr, pr.theta_true))
    times = []
    for it in range(n_iter):
        if it % FIT_LEN == 0:   # fits of FIT_LEN iterations from the initial guess, as on the GPU
            theta, lam = pr.theta_init.copy(), np.array([1e-3])
        t0 = time.perf_counter()
        theta, lam, _ = O.lm_iterate(pr, theta, lam, 1)
        times.append(time.perf_counter() - t0)
    print(json.dumps({"times": times, "n_params": pr.n_params, "n_sources": len(pr.sources),
                      "scale": jacobian_work(full) / jacobian_work(pr),
                      "pixel_scale": sum(im.H * im.W for im in full.images) / sum(im.H * im.W for im in pr.images)}))


def run_oracle(n_iter: int, side: int = SAMPLE_SIDE, threads: int = 1):
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", str(n_iter),
                        "--oracle-side", str(side)],
                       capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle worker failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_line(res, side=SAMPLE_SIDE, threads=1):
    scale = res["scale"]
    t = statistics.mean(res["times"])
    value = 1.0 / (t * scale)
    sample = (f"central {side}x{side} of 2 of the 12 images ({res['n_sources']} sources, {res['n_params']} "
              f"parameters), {len(res['times'])} LM iteration(s) at {t:.2f} s each on {threads} thread(s), scaled to "
              f"the whole workload by its Jacobian work (support pixels x free slots summed over sources) = "
              f"{scale:.0f}x the sample's (pixels: {res['pixel_scale']:.0f}x); the float64 solve grows faster than "
              f"that with the parameter count, so the extrapolation favours the CPU")
    return value, {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the samples go to BENCH_CLOCKS_DIR if set (to keep them), else a temporary directory
        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir(),
                                 f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks(kind="hbm"):
    """Measured peak (HBM GB/s or dense bf16 TFLOP/s burst) and its source."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    key, fallback = ("hbm_gbs", 6800.0) if kind == "hbm" else ("bf16_tflops", 1900.0)
    if os.path.exists(p):
        d = json.load(open(p))
        if key in d:
            return float(d[key]), "measured"
    return fallback, "fallback"


def traffic_from_profiles(kernel, workload=WORKLOAD):
    """Per-launch DRAM bytes of a kernel on a workload from the committed ncu
    summary profiles/dram_traffic_<workload>.txt, or None."""
    p = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        line = line.strip()
        if line and not line.startswith("#") and "=" in line:
            k, v = line.split("=", 1)
            if k.strip() == kernel:
                try:
                    return float(v.split()[0])
                except ValueError:
                    return None
    return None


def measure_pipes(ctx_lib, stream):
    """Throughput of the arithmetic pipes on this GPU (probe kernels of the
    library, ap_measure_pipe): float32 FMA and float64 FMA in TFLOP/s, the
    special-function unit in Tops/s, warp-level TF32 MMA in TFLOP/s; the TF32
    rate of the tcgen05 tensor pipe is the measured bf16 dense rate times the
    nominal tf32 / bf16 ratio 1.1 / 2.25."""
    import ctypes as C
    out = {}
    for name, kind, iters in (("fp32_fma", 0, 4096), ("xu", 1, 2048), ("fp64_fma", 2, 256), ("mma_sync_tf32", 3, 1024)):
        best = None
        for _ in range(3):
            ms, ops = C.c_double(), C.c_double()
            rc = ctx_lib.ap_measure_pipe(kind, iters, C.byref(ms), C.byref(ops), C.c_void_p(stream))
            if rc != 0:
                raise RuntimeError(f"ap_measure_pipe({name}) failed: {rc}")
            r = ops.value / (ms.value * 1e-3) / 1e12
            best = r if best is None else max(best, r)
        out[name] = best
    bf16, src = measured_peaks("bf16")
    out["tf32_tensor"] = bf16 * 1.1 / 2.25
    out["tf32_tensor_source"] = f"{src} bf16 dense {bf16} TFLOP/s x nominal tf32/bf16 ratio 1.1/2.25"
    return out


def gpu_arm(args):
    import numpy as np
    import torch
    from paper_2308_01957_gb300 import api

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    pr = make_problem()
    dimgs = device_problem(pr, dev, local)

    ctx = api.Context("mixed", pr.quad_order, device=local)
    ctx.set_problem(dimgs, pr.sources, pr.n_params)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, steps, warmup, prof_range=False):
        for _ in range(warmup):
            fn()
        if hasattr(fn, "restart"):
            fn.restart()
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        if prof_range:
            # marks the timed steps for a profiler started with collection off
            # (ncu --profile-from-start off); without a profiler it does nothing
            torch.cuda.profiler.start()
        evs = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize(dev)
        if prof_range:
            torch.cuda.profiler.stop()
        if dist:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms

    # ---- LM iterations, mixed precision (the headline): fits of FIT_LEN
    # iterations from the initial guess, one after another ----
    theta_init = torch.tensor(pr.theta_init, dtype=torch.float64, device=dev)
    lm_step = lm_fit(ctx, theta_init)

    with ClockSampler(local) as clk:
        lm_ms = timed(lm_step, args.steps, args.warmup, prof_range=True)
        # chi2 + gradient evaluations, with per-kernel timing inside the library
        th0 = torch.tensor(pr.theta_init, dtype=torch.float64, device=dev)
        out = (torch.empty(ctx.n_groups, dtype=torch.float64, device=dev),
               torch.empty(ctx.n_params, dtype=torch.float64, device=dev))
        ev_ms = timed(eval_cycle(ctx, th0, out), args.eval_steps, args.warmup)
        ctx.set_timing(True)
        timed(eval_cycle(ctx, th0, out), min(args.eval_steps, 8), 0)
        kern = ctx.get_timing()
        # one whole fit with every launch bracketed (no graph): per-kernel times
        lm_step_timed = lm_fit(ctx, theta_init)
        n_lm_t = FIT_LEN
        timed(lm_step_timed, n_lm_t, 0)
        lm_kern, lm_cnt = ctx.get_timing(counts=True)
        ctx.set_timing(False)
    clocks = clk.summary()
    chi2_final = float(ctx.eval(lm_step.state["theta"], grad=False)[0].sum())
    _, _, cg_iters = ctx.state()
    with ClockSampler(local) as clk_p:
        pipes = measure_pipes(ctx.lib, stream.cuda_stream)
    pipes["clocks"] = clk_p.summary()

    # ---- plain float64 GPU form on the same GPU: LM iterations 2.. of a fit
    # (the first one, which also evaluates theta in full, runs untimed) ----
    ctx64 = api.Context("f64", pr.quad_order, device=local)
    ctx64.set_problem(dimgs, pr.sources, pr.n_params)
    lam64 = torch.full((ctx64.n_groups,), 1e-3, dtype=torch.float64, device=dev)
    ctx64.lm_iterate(theta_init.clone(), lam64, 1)
    lm64_ms = timed(lambda: ctx64.lm_continue(1), F64_LM_STEPS, 0)
    out64 = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty(pr.n_params, dtype=torch.float64, device=dev))
    ev64_ms = timed(eval_cycle(ctx64, th0, out64), F64_LM_STEPS, 1)
    # stated relative errors of the mixed form against the float64 form at theta_init
    c32, g32 = ctx.eval(th0)
    c64, g64 = ctx64.eval(th0)
    rel_chi2 = abs(float(c32[0]) - float(c64[0])) / abs(float(c64[0]))
    g32n, g64n = g32.cpu().numpy(), g64.cpu().numpy()
    rel_grad = float(np.max(np.abs(g32n - g64n) / np.maximum(np.abs(g64n), 1e-3 * np.abs(g64n).max())))
    ctx64.close()
    del ctx64
    torch.cuda.empty_cache()

    # ---- end to end through the public API with host buffers ----
    host_data = [im.data.cpu().pin_memory() for im in dimgs]
    host_var = [im.variance.cpu().pin_memory() for im in dimgs]
    host_theta = torch.tensor(pr.theta_init, dtype=torch.float64).pin_memory()
    host_out = torch.empty(pr.n_params + 1, dtype=torch.float64).pin_memory()
    lam_e = torch.tensor([1e-3], dtype=torch.float64, device=dev)

    def e2e_step():
        for im, hd, hv in zip(dimgs, host_data, host_var):
            im.data.copy_(hd, non_blocking=True)
            im.variance.copy_(hv, non_blocking=True)
        th = host_theta.to(dev, non_blocking=True)
        th, lam, chi2, _ = ctx.lm_iterate(th, lam_e, 1)
        host_out[:-1].copy_(th, non_blocking=True)
        host_out[-1:].copy_(chi2, non_blocking=True)

    e2e_steps = max(3, min(args.steps, 20))
    e2e_ms = timed(e2e_step, e2e_steps, min(args.warmup, 3))
    h2d = sum(t.numel() * 4 for t in host_data + host_var) + pr.n_params * 8
    d2h = (pr.n_params + 1) * 8
    del host_data, host_var

    # ---- the other workloads ----
    extra = {}
    if not args.no_extra:
        extra["field_1k"] = measure_extra("field_1k", dev, local, timed, 100, args.warmup, adaptive=True)
        extra["single_sersic"] = measure_extra("single_sersic", dev, local, timed, 20, args.warmup)
        extra["cutouts_256"] = measure_extra("cutouts_256", dev, local, timed, 20, args.warmup)
        extra["crowded_4k"] = measure_extra("crowded_4k", dev, local, timed, 20, 3, f64_lm=False)
        extra["table1_lm_to_convergence"] = [measure_table1(n, dev, local) for n in (1, 16, 64)]

    # ---- gather over ranks (max time) ----
    lm_total, e2e_total = rank_max_totals([lm_ms, e2e_ms], dev, dist)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = job_rate(world, args.steps, lm_total)
    e2e_value = job_rate(world, e2e_steps, e2e_total)
    evals_per_s = 1e3 / statistics.mean(ev_ms)

    # roofline of the dominant kernel of the LM iteration (largest time share
    # over one whole fit)
    share = {k: lm_kern[k] * lm_cnt[k] / n_lm_t for k in lm_kern}
    step_ms = sum(share.values())
    solve = {"iters": int(cg_iters[0]), "nnz": ctx.jtwj_nnz(), "dist": "lm_solve_dist" in lm_kern}
    roofs = {}
    for k in sorted(share, key=share.get, reverse=True):
        # the forward and adjoint brackets run once per chi^2 + gradient
        # evaluation at full work (in the LM step the evaluation at theta of
        # an iteration returns at once), so their duration per launch is the
        # evaluation's; the others run once per LM step
        r = roofline_for(k, (kern if k in kern else lm_kern).get(k), pr, pipes, solve=solve, jcol=ctx.jcol_plan())
        if r and r.get("achieved") is not None:
            r["share_of_step"] = share[k] / step_ms if step_ms else None
            roofs[k] = r
    dom = next(iter(roofs), None)
    roof = roofs.get(dom)
    n_launch_lm, n_launch_eval = launch_counts(ctx)
    f64_lm = 1e3 / statistics.mean(lm64_ms)
    f64_ev = 1e3 / statistics.mean(ev64_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": lm_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 render/conv/Jacobian, f64 chi2/gradient sums/b_n/solve",
        "data": "synthetic (seeded; data = model at true parameters + Gaussian noise of var = model + 1)",
        "config": dict(workload_config(), l2="flushed between timed steps (256 MiB write); inputs (403 MB of data + "
                                             "variance) exceed the 129 MB L2", precision="mixed"),
        "chi2_grad_evals_per_s": evals_per_s,
        "f64_form": {"lm_iters_per_s": f64_lm, "chi2_grad_evals_per_s": f64_ev,
                     "lm_note": f"iterations 2..{F64_LM_STEPS + 1} of a fit from the initial guess"},
        "speedup_vs_f64": {"lm_iters": value / world / f64_lm, "chi2_grad_evals": evals_per_s / f64_ev},
        "rel_error_vs_f64": {"chi2": rel_chi2, "gradient_max": rel_grad},
        "chi2_after_steps": chi2_final,
        "cg_iterations_last_solve": int(cg_iters[0]),
        "jacobian_convolution": dict(zip(("mode", "ms_direct", "ms_fft"), ctx.jcol_mode())),
        "kernel_ms_chi2_grad_eval": kern,
        "kernel_ms_per_lm_step": share,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": n_launch_lm * args.steps,
        "launches_per_step": n_launch_lm,
        "launches_per_chi2_grad_eval": n_launch_eval,
        "roofline": roof,
        "rooflines_by_kernel": roofs,
        "measured_pipes": pipes,
        "clocks": clocks,
        "extra_workloads": extra,
    }
    if not args.no_cpu_baseline and world == 1:
        res = run_oracle(1, threads=1)
        _, cpu1 = oracle_line(res, threads=1)
        nproc = os.cpu_count() or 1
        resn = run_oracle(1, threads=nproc)
        _, cpun = oracle_line(resn, threads=nproc)
        line["cpu_baseline"] = cpun if cpun["value"] > cpu1["value"] else cpu1
        line["cpu_baseline_by_threads"] = {"1": cpu1["value"], str(nproc): cpun["value"]}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def device_problem(pr, dev, local):
    """Device images with data made by the library's float64 render at
    theta_true plus the workload's seeded noise."""
    import numpy as np
    from paper_2308_01957_gb300 import api
    from synthetic.problem import attach_data
    for im in pr.images:   # provisional planes so the context can be built
        im.data = np.zeros((im.H, im.W), np.float32)
        im.variance = np.ones((im.H, im.W), np.float32)
    tmp = api.Context("f64", pr.data_quad_order or pr.quad_order, device=local)
    tmp.set_problem(api.to_device_images(pr.images, dev), pr.sources, pr.n_params)
    models = [m.cpu().numpy() for m in tmp.render(pr.theta_true)]
    tmp.close()
    attach_data(pr, models)
    return api.to_device_images(pr.images, dev)


def measure_extra(name, dev, local, timed, steps, warmup, f64_lm=True, adaptive=False):
    """LM iterations / s and chi^2 + gradient evaluations / s of another
    workload in the mixed form, and the same for the float64 form (its LM
    iterations only when f64_lm: on the largest fields one float64 iteration
    takes seconds); with adaptive, the adaptive-integration figures too."""
    import statistics
    import torch
    from paper_2308_01957_gb300 import api
    from synthetic import configs
    pr = configs.WORKLOADS[name]()
    dimgs = device_problem(pr, dev, local)
    out = {"note": pr.note, "groups": pr.n_groups, "params": pr.n_params,
           "pixels": int(sum(im.H * im.W for im in pr.images))}
    for prec in ("mixed", "f64"):
        ctx = api.Context(prec, pr.quad_order, device=local)
        ctx.set_problem(dimgs, pr.sources, pr.n_params)
        n = steps if prec == "mixed" else max(1, min(steps // 4, 20))
        res = {}
        if prec == "mixed" or f64_lm:
            lm_step = lm_fit(ctx, torch.tensor(pr.theta_init, dtype=torch.float64, device=dev))
            lm_ms = timed(lm_step, n, warmup if prec == "mixed" else 1)
            res["lm_iters_per_s"] = 1e3 / statistics.mean(lm_ms)
            res["ms_per_lm_iter"] = statistics.mean(lm_ms)
            if prec == "mixed":
                mode, ms_d, ms_f = ctx.jcol_mode()
                res["jacobian_convolution"] = {"mode": mode, "ms_direct": ms_d, "ms_fft": ms_f}
                # per-kernel breakdown over one whole fit (event-bracketed, un-graphed)
                ctx.set_timing(True)
                ctx.get_timing()
                t_step = lm_fit(ctx, torch.tensor(pr.theta_init, dtype=torch.float64, device=dev))
                for _ in range(FIT_LEN):
                    t_step()
                torch.cuda.synchronize()
                avg, cnt = ctx.get_timing(counts=True)
                res["kernel_ms_per_lm_step"] = {k: avg[k] * cnt[k] / FIT_LEN for k in avg}
                res["cg_iterations"] = [int(x) for x in ctx.state()[2][:4]]
                ctx.set_timing(False)
        th0 = torch.tensor(pr.theta_init, dtype=torch.float64, device=dev)
        o = (torch.empty(ctx.n_groups, dtype=torch.float64, device=dev),
             torch.empty(ctx.n_params, dtype=torch.float64, device=dev))
        ev_ms = timed(eval_cycle(ctx, th0, o), n, 1)
        res["chi2_grad_evals_per_s"] = 1e3 / statistics.mean(ev_ms)
        if adaptive and prec == "mixed":
            out["adaptive_integration"] = measure_adaptive(ctx, th0, timed, 50, warmup)
        out[prec] = res
        ctx.close()
    out["speedup_vs_f64"] = {k: out["mixed"][k] / out["f64"][k] for k in ("lm_iters_per_s", "chi2_grad_evals_per_s")
                             if k in out["f64"]}
    del dimgs
    torch.cuda.empty_cache()
    return out


def measure_table1(n_sersic, dev, local, max_iter=100, rtol=1e-6):
    """The paper's GPU benchmark (Table 1): n_sersic overlapping Sersics on a
    1000 x 1000 image, fitted by LM from the perturbed start until an accepted
    iteration lowers chi^2 by less than rtol (relative), at most max_iter
    iterations; every iteration timed with CUDA events.  Returns the time and
    the iterations to convergence, the mean time per iteration and the final
    chi^2 per pixel."""
    import numpy as np
    import torch
    from paper_2308_01957_gb300 import api
    from synthetic import configs
    pr = configs.table1(n_sersic)
    dimgs = device_problem(pr, dev, local)
    ctx = api.Context("mixed", pr.quad_order, device=local)
    ctx.set_problem(dimgs, pr.sources, pr.n_params)
    stream = torch.cuda.current_stream(dev)
    th0 = torch.tensor(pr.theta_init, dtype=torch.float64, device=dev)
    lam = torch.full((1,), 1e-3, dtype=torch.float64, device=dev)
    ctx.lm_iterate(th0.clone(), lam.clone(), 1)   # warm-up (graph capture)
    torch.cuda.synchronize(dev)
    evs, chis, accs = [], [], []
    for it in range(max_iter):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        if it == 0:
            _, _, chi2, _ = ctx.lm_iterate(th0.clone(), lam.clone(), 1)
        else:
            _, _, chi2, _ = ctx.lm_continue(1)
        b.record(stream)
        evs.append((a, b))
        chis.append(chi2.clone())
    torch.cuda.synchronize(dev)
    ms = [a.elapsed_time(b) for a, b in evs]
    c = [float(x[0]) for x in chis]
    c0 = float(ctx.eval(th0, grad=False)[0][0])
    prev, k_conv = c0, max_iter
    for k, ck in enumerate(c):
        if ck < prev and (prev - ck) < rtol * prev:
            k_conv = k + 1
            break
        prev = min(prev, ck)
    out = {"n_sersic": n_sersic, "params": pr.n_params, "iterations_to_convergence": k_conv,
           "ms_to_convergence": float(sum(ms[:k_conv])), "ms_per_lm_iter": float(np.mean(ms)),
           "chi2_per_pixel_start": c0 / 1e6, "chi2_per_pixel_final": c[k_conv - 1] / 1e6,
           "criterion": f"first accepted iteration lowering chi2 by less than {rtol} relative (cap {max_iter})"}
    ctx.close()
    del dimgs
    torch.cuda.empty_cache()
    return out


def measure_adaptive(ctx, theta, timed, steps, warmup, tol=0.01):
    """chi^2 evaluations / s of the model sampled by adaptive pixel
    integration (budget tol) against the fixed order-3 rule on the same
    problem, how many samples end at each level, the quadrature nodes each
    form evaluates, and the kernel time per adaptive evaluation."""
    import statistics
    import torch
    chi2 = torch.empty(ctx.n_groups, dtype=torch.float64, device=theta.device)
    cnt = ctx.eval_adaptive(theta, tol=tol, counts=True)["counts"]
    n_samp = int(cnt[:4].sum())
    # nodes per sample: midpoint 1; orders 3 + 2: 13; 25 sub-pixels x (25 + 16); 25 x 49 per sub-pixel split again
    nodes = int(cnt[0] + 14 * cnt[1] + (14 + 25 * 41) * (cnt[2] + cnt[3]) + 25 * 49 * cnt[4])
    ad_ms = timed(lambda: ctx.eval_adaptive(theta, tol=tol), steps, warmup)
    fx_ms = timed(lambda: ctx.eval(theta, grad=False, out=(chi2, None)), steps, warmup)
    ctx.set_timing(True)
    ctx.get_timing()
    ctx.eval_adaptive(theta, tol=tol)
    torch.cuda.synchronize()
    kern = ctx.get_timing()
    ctx.set_timing(False)
    samp_ms = kern.get("adaptive_sampling", 0.0)
    return {"tol": tol, "samples": n_samp,
            "levels": {"midpoint": int(cnt[0]), "order3": int(cnt[1]), "split_order5": int(cnt[2]),
                       "split_again_order7": int(cnt[3]), "sub_pixels_split_again": int(cnt[4])},
            "nodes_adaptive": nodes, "nodes_fixed_order3": 9 * n_samp,
            "chi2_evals_per_s_adaptive": 1e3 / statistics.mean(ad_ms),
            "chi2_evals_per_s_fixed_order3": 1e3 / statistics.mean(fx_ms),
            "kernel_ms_per_eval": kern,
            "sampling_nodes_per_s": nodes / (samp_ms * 1e-3) if samp_ms > 0 else None}


def launch_counts(ctx):
    """Kernels per LM iteration (nodes of the captured graph) and per eval."""
    import ctypes as C
    n_it, n_ev = C.c_int(), C.c_int()
    ctx.lib.ap_get_launch_count(ctx.h, C.byref(n_it), C.byref(n_ev))
    return n_it.value, n_ev.value


def _support(s, im, h):
    """Sampling box and Jacobian support (image pixels) of a source."""
    x0, x1, y0, y1 = s.win
    x0, x1, y0, y1 = max(x0, 0), min(x1, im.W), max(y0, 0), min(y1, im.H)
    if x0 >= x1 or y0 >= y1:
        return 0, 0
    hh = h if s.psf_convolve else 0
    box = (min(y1 + hh, im.H + hh) - max(y0 - hh, -hh)) * (min(x1 + hh, im.W + hh) - max(x0 - hh, -hh))
    sup = (min(y1 + 2 * hh, im.H) - max(y0 - 2 * hh, 0)) * (min(x1 + 2 * hh, im.W) - max(x0 - 2 * hh, 0))
    return box, sup


def roofline_for(name, ms, pr, pipes, solve=None, jcol=None):
    """Roofline of one kernel from its CUDA-event duration (average per
    launch), against the pipe rates measured on this GPU (measure_pipes).
    Algorithmic work per launch, summed over the problem's images:
    * forward_conv_chi2 / adjoint_conv: 2 K^2 flops per output pixel (image
      pixels / galaxy-layer pixels), FP32 pipe;
    * jacobian_columns: direct mode, 2 K^2 flops per Jacobian-support pixel
      per free slot of each convolved source; FFT mode, per N x N block a
      forward and an inverse real-input 2-D FFT (2 x 2.5 N^2 log2 N^2 flops)
      and the spectrum product (6 N (N/2+1)); FP32 pipe;
    * render / render_adjoint: transcendental (XU) operations per quadrature
      node (Sersic 3, Moffat 2, Gaussian 1) over the sampling boxes;
    * jtwj_gram: 3 x 2 x 256 x C(C+1)/2 flops per 16x16 tile with C free
      columns (3xTF32), TF32 tensor rate;
    * lm_solve / lm_solve_dist: float64 flops of the PCG per launch, CG
      iterations x (2 nnz of J^T W J + 2 m^2 per preconditioner block of m
      parameters + 14 per parameter) plus the block factorisations (2 m^3);
      FP64 pipe."""
    if not name or not ms:
        return None
    import numpy as np
    out = {"kernel": name, "traffic": traffic_from_profiles(name)}

    def h_of(im):
        return 0 if im.psf is None else (im.psf.shape[0] - 1) // 2

    def done(bound, flops, peak, unit, peak_source, work):
        ach = flops / (ms * 1e-3) / 1e12
        out.update(bound=bound, achieved=ach, peak=peak, unit=unit, frac=ach / peak, peak_source=peak_source,
                   work=work)
        return out

    fp32 = (pipes["fp32_fma"], "measured on this GPU (float32 FMA probe, ap_measure_pipe)")
    if name == "jacobian_columns" and jcol and jcol[0] == "fft":
        flops = sum(nb * (2 * 2.5 * n * n * math.log2(n * n) + 6.0 * n * (n // 2 + 1))
                    for n, nb in ((64, jcol[3]), (128, jcol[4])))
        return done("alu", flops, fp32[0], "TFLOP/s", fp32[1],
                    f"FFT mode: {jcol[3]} blocks of 64^2 and {jcol[4]} of 128^2, forward + inverse real-input 2-D FFT "
                    "and the spectrum product per block")
    if name in ("forward_conv_chi2", "adjoint_conv", "jacobian_columns"):
        flops, npx = 0.0, 0
        for ii, im in enumerate(pr.images):
            if im.psf is None:
                continue
            K, h = im.psf.shape[0], h_of(im)
            if name == "forward_conv_chi2":
                n = im.H * im.W
            elif name == "adjoint_conv":
                n = (im.H + 2 * h) * (im.W + 2 * h)
            else:
                n = sum(_support(s, im, h)[1] * sum(1 for k in range(8) if s.pidx[k] >= 0)
                        for s in pr.sources if s.psf_convolve and s.image == ii)
            flops += 2.0 * K * K * n
            npx += n
        return done("alu", flops, fp32[0], "TFLOP/s", fp32[1], f"2 K^2 flops per output pixel, {npx} output pixels")
    if name in ("render", "render_adjoint"):
        xu = 0
        for s in pr.sources:
            im = pr.images[s.image]
            h = h_of(im) if s.psf_convolve else 0
            xu += _support(s, im, h)[0] * pr.quad_order ** 2 * {0: 3, 1: 3, 2: 1, 3: 2}.get(s.type, 0)
        return done("alu", xu, pipes["xu"], "Tops/s (XU)", "measured on this GPU (ex2/lg2 probe, ap_measure_pipe)",
                    "transcendentals per quadrature node: Sersic 3 (lg2, 2 ex2), Moffat 2, Gaussian 1")
    if name == "jtwj_gram":
        flops, nbytes = 0.0, 0.0
        for ii, im in enumerate(pr.images):
            h = h_of(im)
            cols = np.zeros(((im.H + 15) // 16, (im.W + 15) // 16))
            for s in pr.sources:
                if s.image != ii:
                    continue
                x0, x1, y0, y1 = s.win
                hh = 2 * h if s.psf_convolve else 0
                r0, r1 = max(y0 - hh, 0), min(y1 + hh, im.H)
                c0, c1 = max(x0 - hh, 0), min(x1 + hh, im.W)
                if r0 < r1 and c0 < c1:
                    cols[r0 // 16:(r1 - 1) // 16 + 1, c0 // 16:(c1 - 1) // 16 + 1] += \
                        sum(1 for k in range(8) if s.pidx[k] >= 0)
            flops += float(np.sum(3 * 2 * 256 * cols * (cols + 1) / 2))
            nbytes += float(np.sum(cols * 256 * 4 + cols * (cols + 1) / 2 * 8 * 2))
        # the contraction's intensity (~0.75 C flop per byte of columns) is far
        # below the TF32 ridge, so its roofline is HBM: the columns read once
        # (C x 256 x 4 bytes per tile) and the pair blocks written and read back
        # once (C (C+1) / 2 x 8 bytes each way); the tensor pipe's share is kept
        hbm, src = measured_peaks("hbm")
        ach_t = flops / (ms * 1e-3) / 1e12
        ach = nbytes / (ms * 1e-3) / 1e9
        out.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                   peak_source=f"{src} HBM copy (MEASURED_PEAKS.json)",
                   work="Jacobian columns C x 1 KB per 16 x 16 tile read once, C(C+1)/2 float64 pair entries "
                        "written and read back once")
        out["tensor"] = {"achieved_tflops": ach_t, "peak_tflops": pipes["tf32_tensor"],
                         "frac": ach_t / pipes["tf32_tensor"], "peak_source": pipes["tf32_tensor_source"],
                         "work": "3xTF32: three TF32 products per column pair over 256 pixels per tile"}
        return out
    if name in ("lm_solve", "lm_solve_dist") and solve:
        if name == "lm_solve" and solve.get("dist"):
            return None   # the group is solved by the distributed PCG; lm_solve launches no work here
        blocks = []
        for s in pr.sources:
            f = sum(1 for k in range(8) if s.pidx[k] >= 0)
            while f > 0:
                blocks.append(min(f, 8))
                f -= 8
        m2 = sum(m * m for m in blocks)
        m3 = sum(m ** 3 for m in blocks)
        flops = solve["iters"] * (2.0 * solve["nnz"] + 2.0 * m2 + 14.0 * pr.n_params) + 2.0 * m3
        return done("fp64", flops, pipes["fp64_fma"], "TFLOP/s",
                    "measured on this GPU (float64 FMA probe, ap_measure_pipe)",
                    f"{solve['iters']} CG iterations x (2 x {solve['nnz']} nnz + block products), block factors")
    return None


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # a bounded sample per step: the central crop of two images shrinks so
    # that warmup + steps oracle iterations stay near two and a half minutes
    # (about 13 s per iteration on the 256 x 256 sample, one thread)
    n = args.warmup + args.steps
    side = int(min(SAMPLE_SIDE, max(96, SAMPLE_SIDE * math.sqrt(150.0 / (13.0 * max(n, 1))))) // 16 * 16)
    res = run_oracle(n, side)
    res["times"] = res["times"][args.warmup:]
    value, cpu = oracle_line(res, side)
    t = statistics.mean(res["times"]) * res["scale"]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": dict(workload_config(), precision="f64 CPU oracle"),
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def profile_arm(args):
    """A few LM iterations of one workload for profilers: the iterations after
    the warm-up are bracketed by cudaProfilerStart/Stop (ncu
    --profile-from-start off captures only those).  --profile joint_12x2k_crop
    is the central 512 x 512 of two images of the joint fit (the size of an
    ncu --set full capture)."""
    import torch
    from paper_2308_01957_gb300 import api
    from synthetic import configs
    dev = torch.device("cuda", 0)
    if args.profile == "joint_12x2k_crop":
        pr = crop_problem(configs.joint(), SAMPLE_IMAGES, 768, 768, 512, 512)
    else:
        pr = configs.WORKLOADS[args.profile]()
    dimgs = device_problem(pr, dev, 0)
    ctx = api.Context("mixed", pr.quad_order, device=0)
    ctx.set_problem(dimgs, pr.sources, pr.n_params)
    step = lm_fit(ctx, torch.tensor(pr.theta_init, dtype=torch.float64, device=dev))
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    mode, _, _, n64, n128 = ctx.jcol_plan()
    print(json.dumps({"profile": args.profile, "params": pr.n_params, "lm_iterations": args.steps,
                      "launches_per_step": launch_counts(ctx)[0], "jacobian_convolution": mode,
                      "fft_blocks_64": n64, "fft_blocks_128": n128, "status": ctx.status()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--eval-steps", type=int, default=50)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads (cutouts, 4k field, joint fit)")
    ap.add_argument("--oracle-worker", type=int, default=0)
    ap.add_argument("--oracle-side", type=int, default=SAMPLE_SIDE)
    ap.add_argument("--profile", default=None, help="run LM iterations of one workload for a profiler and exit")
    args = ap.parse_args()
    if args.profile:
        profile_arm(args)
        return
    if args.oracle_worker:
        oracle_worker(args.oracle_worker, args.oracle_side)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    gpu_arm(args)


if __name__ == "__main__":
    main()
