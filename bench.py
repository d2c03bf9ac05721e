"""Benchmark of the chi^2 forward-modelling path on the 1024x1024 field
(50 Sersic galaxies + 200 Moffat point sources, 25x25 Moffat PSF, Q = 3).

A step is one Levenberg-Marquardt iteration: chi^2 + adjoint gradient at
theta, the Jacobian / J^T W J build, the damped float64 solve, chi^2 at the
trial point and the on-device accept -- every step of the path.  The line also
reports chi^2 + gradient evaluations per second and both numbers for the plain
float64 GPU form on the same GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (single thread) and prints the same metric.
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
WORKLOAD = "field_1k"
SAMPLE_SIDE = 512          # oracle sample: a 512x512 crop (1/4 of the field, same source density)
FIT_LEN = 20               # timed LM iterations restart the fit from the initial guess every FIT_LEN steps


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
    return {"workload": "field_1k: 1024x1024 FP32 image, 50 Sersic + 200 Moffat (beta 3, FWHM 3 px), plane sky, "
                        "25x25 Moffat PSF, 3x3 Gauss-Legendre per pixel, var = model + 1, 953 parameters",
            "step": "one LM iteration (chi2+adjoint gradient, J^T W J, damped FP64 solve, trial chi2, accept)",
            "fits": f"timed iterations form fits of {FIT_LEN} LM iterations, each from the initial guess (lambda 1e-3)"}


# ---------------------------------------------------------------------------
# problem set-up (inputs only)
# ---------------------------------------------------------------------------

def make_problem():
    from synthetic import configs
    return configs.field_1k()


def crop_problem(pr, side):
    """The workload restricted to its lower-left side x side pixels: sources
    whose window meets the crop, windows clipped, parameters renumbered."""
    import numpy as np
    from synthetic.problem import ImageSpec, Problem, SourceSpec
    im = pr.images[0]
    new_im = ImageSpec(H=side, W=side, A=im.A, origin=im.origin, psf=im.psf,
                       mask=None if im.mask is None else im.mask[:side, :side].copy(), group=0)
    keep, idx_map = [], {}
    for s in pr.sources:
        x0, x1, y0, y1 = s.win
        x0, x1, y0, y1 = max(x0, 0), min(x1, side), max(y0, 0), min(y1, side)
        if x0 >= x1 or y0 >= y1:
            continue
        pidx = s.pidx.copy()
        for k in range(8):
            if pidx[k] >= 0:
                pidx[k] = idx_map.setdefault(int(pidx[k]), len(idx_map))
        keep.append(SourceSpec(s.type, 0, (x0, x1, y0, y1), s.psf_convolve, pidx, s.pfix.copy()))
    order = sorted(idx_map, key=idx_map.get)
    return Problem(pr.name + f"_crop{side}", [new_im], keep, len(order), pr.theta_true[order], pr.theta_init[order],
                   quad_order=pr.quad_order, noise=[pr.noise[0][:side, :side].copy()], var_floor=pr.var_floor)


# ---------------------------------------------------------------------------
# CPU oracle leg (runs in a fresh single-threaded interpreter)
# ---------------------------------------------------------------------------

def oracle_worker(n_iter: int, side: int = SAMPLE_SIDE):
    """Time the oracle, as it stands, on a side x side crop: n_iter LM iterations."""
    from oracle import astrophot_oracle as O
    from synthetic.problem import attach_data
    import numpy as np
    pr = crop_problem(make_problem(), side)
    attach_data(pr, O.model_images(pr, pr.theta_true))
    times = []
    for it in range(n_iter):
        if it % FIT_LEN == 0:   # fits of FIT_LEN iterations from the initial guess, as on the GPU
            theta, lam = pr.theta_init.copy(), np.array([1e-3])
        t0 = time.perf_counter()
        theta, lam, _ = O.lm_iterate(pr, theta, lam, 1)
        times.append(time.perf_counter() - t0)
    print(json.dumps({"times": times, "n_params": pr.n_params, "n_sources": len(pr.sources)}))


def run_oracle(n_iter: int, side: int = SAMPLE_SIDE):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", str(n_iter),
                        "--oracle-side", str(side)],
                       capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle worker failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_line(res, side=SAMPLE_SIDE):
    scale = (1024 * 1024) / (side * side)
    t = statistics.mean(res["times"])
    value = 1.0 / (t * scale)
    sample = (f"{side}x{side} crop of the field ({res['n_sources']} sources, {res['n_params']} parameters), "
              f"{len(res['times'])} LM iteration(s) at {t:.2f} s each, scaled by the area ratio {scale:g} to the full field")
    return value, {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}


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


def traffic_from_profiles(kernel):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, or None."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
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


def gpu_arm(args):
    import numpy as np
    import torch
    from paper_2308_01957_gb300 import api
    from synthetic.problem import attach_data

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
        timed(eval_cycle(ctx, th0, out), args.eval_steps, 0)
        kern = ctx.get_timing()
        # the same LM iterations with every launch bracketed (no graph)
        lm_step_timed = lm_fit(ctx, theta_init)
        n_lm_t = max(FIT_LEN, args.steps // 4)
        timed(lm_step_timed, n_lm_t, 0)
        lm_kern, lm_cnt = ctx.get_timing(counts=True)
        ctx.set_timing(False)
    clocks = clk.summary()
    chi2_final = float(ctx.eval(lm_step.state["theta"], grad=False)[0].sum())
    _, _, cg_iters = ctx.state()

    # ---- plain float64 GPU form on the same GPU ----
    ctx64 = api.Context("f64", pr.quad_order, device=local)
    ctx64.set_problem(dimgs, pr.sources, pr.n_params)
    lm_step64 = lm_fit(ctx64, theta_init)
    n64 = max(FIT_LEN, args.steps // 4)
    lm64_ms = timed(lm_step64, n64, 1)
    out64 = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty(pr.n_params, dtype=torch.float64, device=dev))
    ev64_ms = timed(eval_cycle(ctx64, th0, out64), n64, 1)
    # stated relative errors of the mixed form against the float64 form at theta_init
    c32, g32 = ctx.eval(th0)
    c64, g64 = ctx64.eval(th0)
    rel_chi2 = abs(float(c32[0]) - float(c64[0])) / abs(float(c64[0]))
    g32n, g64n = g32.cpu().numpy(), g64.cpu().numpy()
    rel_grad = float(np.max(np.abs(g32n - g64n) / np.maximum(np.abs(g64n), 1e-3 * np.abs(g64n).max())))
    ctx64.close()

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

    e2e_ms = timed(e2e_step, args.steps, args.warmup)
    h2d = sum(t.numel() * 4 for t in host_data + host_var) + pr.n_params * 8
    d2h = (pr.n_params + 1) * 8

    # ---- the batched-cutouts workload: 256 independent fits per launch ----
    extra = {}
    if not args.no_extra:
        extra["single_sersic"] = measure_extra("single_sersic", dev, local, timed, 20, args.warmup)
        extra["cutouts_256"] = measure_extra("cutouts_256", dev, local, timed, min(max(3, args.steps // 2), 20),
                                             args.warmup)
        extra["crowded_4k"] = measure_extra("crowded_4k", dev, local, timed, 3, 1, f64_lm=False)
        extra["joint_12x2k"] = measure_extra("joint_12x2k", dev, local, timed, 3, 1, f64_lm=False)
        extra["adaptive_integration_field_1k"] = measure_adaptive(ctx, th0, timed, 50, args.warmup)

    # ---- gather over ranks (max time) ----
    lm_total, e2e_total = rank_max_totals([lm_ms, e2e_ms], dev, dist)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = job_rate(world, args.steps, lm_total)
    e2e_value = job_rate(world, args.steps, e2e_total)
    evals_per_s = 1e3 / statistics.mean(ev_ms)

    # roofline of the dominant kernel of the LM iteration (largest time share)
    share = {k: lm_kern[k] * lm_cnt[k] / n_lm_t for k in lm_kern}
    step_ms = sum(share.values())
    dom = max(share, key=share.get) if share else None
    roof = roofline_for(dom, lm_kern.get(dom) if dom else None, pr,
                        solve={"iters": int(cg_iters[0]), "nnz": ctx.jtwj_nnz(), "dist": "lm_solve_dist" in lm_kern},
                        jcol=ctx.jcol_plan())
    if roof is not None:
        roof["share_of_step"] = share[dom] / step_ms if step_ms else None
    # the same figures for every kernel of the step that has a roofline
    other_roofs = {}
    for k in sorted(share, key=share.get, reverse=True):
        r = roofline_for(k, lm_kern.get(k), pr, solve={"iters": int(cg_iters[0]), "nnz": ctx.jtwj_nnz(),
                                                        "dist": "lm_solve_dist" in lm_kern}, jcol=ctx.jcol_plan())
        if r and r.get("achieved") is not None:
            other_roofs[k] = {"bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"], "unit": r["unit"],
                              "frac": r["frac"], "share_of_step": share[k] / step_ms if step_ms else None}
    n_launch_lm, n_launch_eval = launch_counts(ctx)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": lm_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 render/conv/Jacobian, f64 chi2/gradient sums/b_n/solve",
        "data": "synthetic (seeded; data = model at true parameters + Gaussian noise of var = model + 1)",
        "config": dict(workload_config(), l2="flushed between timed steps (256 MiB write)", precision="mixed"),
        "chi2_grad_evals_per_s": evals_per_s,
        "f64_form": {"lm_iters_per_s": 1e3 / statistics.mean(lm64_ms), "chi2_grad_evals_per_s": 1e3 / statistics.mean(ev64_ms)},
        "speedup_vs_f64": {"lm_iters": value / world / (1e3 / statistics.mean(lm64_ms)),
                           "chi2_grad_evals": evals_per_s / (1e3 / statistics.mean(ev64_ms))},
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
        "rooflines_by_kernel": other_roofs,
        "clocks": clocks,
        "extra_workloads": extra,
    }
    if not args.no_cpu_baseline and world == 1:
        res = run_oracle(1)
        _, cpu = oracle_line(res)
        line["cpu_baseline"] = cpu
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
    tmp = api.Context("f64", pr.quad_order, device=local)
    tmp.set_problem(api.to_device_images(pr.images, dev), pr.sources, pr.n_params)
    models = [m.cpu().numpy() for m in tmp.render(pr.theta_true)]
    tmp.close()
    attach_data(pr, models)
    return api.to_device_images(pr.images, dev)


def measure_extra(name, dev, local, timed, steps, warmup, f64_lm=True):
    """LM iterations / s and chi^2 + gradient evaluations / s of another
    workload in the mixed form, and the same for the float64 form (its LM
    iterations only when f64_lm: on the largest fields one float64 iteration
    takes many seconds)."""
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
        n = steps if prec == "mixed" else max(1, steps // 3)
        res = {}
        if prec == "mixed" or f64_lm:
            lm_step = lm_fit(ctx, torch.tensor(pr.theta_init, dtype=torch.float64, device=dev))
            lm_ms = timed(lm_step, n, warmup if prec == "mixed" else 1)
            res["lm_iters_per_s"] = 1e3 / statistics.mean(lm_ms)
            res["ms_per_lm_iter"] = statistics.mean(lm_ms)
            if prec == "mixed":
                mode, ms_d, ms_f = ctx.jcol_mode()
                res["jacobian_convolution"] = {"mode": mode, "ms_direct": ms_d, "ms_fft": ms_f}
                # per-kernel breakdown of one more iteration (event-bracketed, un-graphed)
                ctx.set_timing(True)
                ctx.get_timing()
                lm_step()
                torch.cuda.synchronize()
                avg, cnt = ctx.get_timing(counts=True)
                res["kernel_ms_per_lm_step"] = {k: avg[k] * cnt[k] for k in avg}
                res["cg_iterations"] = [int(x) for x in ctx.state()[2][:4]]
                ctx.set_timing(False)
        th0 = torch.tensor(pr.theta_init, dtype=torch.float64, device=dev)
        o = (torch.empty(ctx.n_groups, dtype=torch.float64, device=dev),
             torch.empty(ctx.n_params, dtype=torch.float64, device=dev))
        ev_ms = timed(eval_cycle(ctx, th0, o), n, 1)
        res["chi2_grad_evals_per_s"] = 1e3 / statistics.mean(ev_ms)
        out[prec] = res
        ctx.close()
    out["speedup_vs_f64"] = {k: out["mixed"][k] / out["f64"][k] for k in ("lm_iters_per_s", "chi2_grad_evals_per_s")
                             if k in out["f64"]}
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


def roofline_for(name, ms, pr, solve=None, jcol=None):
    """Roofline of one kernel from its CUDA-event duration (average per
    launch).  Algorithmic work per launch:
    * forward_conv_chi2 / adjoint_conv: 2 K^2 flops per output pixel (FP32
      pipe; peak = SMs x 128 lanes x 2 x max clock);
    * jacobian_columns: direct mode, 2 K^2 flops per Jacobian-support pixel
      per free slot of each convolved source (FP32 pipe); FFT mode, per N x N
      block a forward and an inverse real-input 2-D FFT (2 x 2.5 N^2 log2 N^2
      flops) and the spectrum product (6 N (N/2+1));
    * render / render_adjoint: transcendental (XU) operations per quadrature
      node (Sersic 3, Moffat 2, Gaussian 1); peak = SMs x 16 x max clock;
    * jtwj_gram: 3 x 2 x 256 x C(C+1)/2 flops per 16x16 tile with C free
      columns (3xTF32 on the tensor pipe); peak = measured bf16 x 1.1/2.25;
    * lm_solve / lm_solve_dist: float64 flops of the PCG per launch, CG
      iterations x (2 nnz of J^T W J + 2 m^2 per preconditioner block of m
      parameters + 14 per parameter) plus the block factorisations
      (2 m^3); float64 pipe, peak 1.25 TFLOP/s nominal."""
    if not name or not ms:
        return None
    import numpy as np
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    clock = 2070e6
    im = pr.images[0]
    K = im.psf.shape[0]
    h = (K - 1) // 2
    fp32_peak = sms * 128 * 2 * clock / 1e12
    xu_peak = sms * 16 * clock / 1e12
    out = {"kernel": name, "traffic": traffic_from_profiles(name)}
    if name == "jacobian_columns" and jcol and jcol[0] == "fft":
        flops = sum(nb * (2 * 2.5 * n * n * math.log2(n * n) + 6.0 * n * (n // 2 + 1))
                    for n, nb in ((64, jcol[3]), (128, jcol[4])))
        ach = flops / (ms * 1e-3) / 1e12
        out.update(bound="alu", achieved=ach, peak=fp32_peak, unit="TFLOP/s", frac=ach / fp32_peak,
                   peak_source=f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                   work=f"FFT mode: {jcol[3]} blocks of 64^2 and {jcol[4]} of 128^2, forward + inverse real-input "
                        "2-D FFT and the spectrum product per block")
        return out
    if name in ("forward_conv_chi2", "adjoint_conv", "jacobian_columns"):
        if name == "forward_conv_chi2":
            npx = im.H * im.W
        elif name == "adjoint_conv":
            npx = (im.H + 2 * h) * (im.W + 2 * h)
        else:
            npx = sum(_support(s, im, h)[1] * sum(1 for k in range(8) if s.pidx[k] >= 0)
                      for s in pr.sources if s.psf_convolve)
        flops = 2.0 * K * K * npx
        ach = flops / (ms * 1e-3) / 1e12
        out.update(bound="alu", achieved=ach, peak=fp32_peak, unit="TFLOP/s", frac=ach / fp32_peak,
                   peak_source=f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                   work=f"2 K^2 flops per output pixel, K={K}, {npx} output pixels")
        return out
    if name in ("render", "render_adjoint"):
        xu = sum(_support(s, im, h)[0] * pr.quad_order ** 2 * {0: 3, 1: 3, 2: 1, 3: 2}.get(s.type, 0)
                 for s in pr.sources)
        ach = xu / (ms * 1e-3) / 1e12
        out.update(bound="alu", achieved=ach, peak=xu_peak, unit="Tops/s (XU)", frac=ach / xu_peak,
                   peak_source=f"derived: {sms} SMs x 16 XU lanes x 2070 MHz",
                   work="transcendentals per quadrature node: Sersic 3 (lg2, 2 ex2), Moffat 2, Gaussian 1")
        return out
    if name == "jtwj_gram":
        cols = np.zeros(((im.H + 15) // 16, (im.W + 15) // 16))
        for s in pr.sources:
            x0, x1, y0, y1 = s.win
            hh = 2 * h if s.psf_convolve else 0
            r0, r1 = max(y0 - hh, 0), min(y1 + hh, im.H)
            c0, c1 = max(x0 - hh, 0), min(x1 + hh, im.W)
            if r0 < r1 and c0 < c1:
                cols[r0 // 16:(r1 - 1) // 16 + 1, c0 // 16:(c1 - 1) // 16 + 1] += sum(1 for k in range(8) if s.pidx[k] >= 0)
        flops = float(np.sum(3 * 2 * 256 * cols * (cols + 1) / 2))
        ach = flops / (ms * 1e-3) / 1e12
        bf16, _ = measured_peaks(kind="bf16")
        peak = bf16 * 1.1 / 2.25
        out.update(bound="tensor", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                   peak_source="measured bf16 dense (MEASURED_PEAKS.json) x nominal tf32/bf16 ratio 1.1/2.25",
                   work="3xTF32: three m16n8k8 MMAs per product over 256 pixels per tile, C(C+1)/2 column pairs")
        return out
    if name == "lm_solve" and solve and solve.get("dist"):
        return None   # the group is solved by the distributed PCG; lm_solve launches no work here
    if name in ("lm_solve", "lm_solve_dist") and solve:
        blocks = []
        for s in pr.sources:
            f = sum(1 for k in range(8) if s.pidx[k] >= 0)
            while f > 0:
                blocks.append(min(f, 8))
                f -= 8
        m2 = sum(m * m for m in blocks)
        m3 = sum(m ** 3 for m in blocks)
        flops = solve["iters"] * (2.0 * solve["nnz"] + 2.0 * m2 + 14.0 * pr.n_params) + 2.0 * m3
        ach = flops / (ms * 1e-3) / 1e12
        out.update(bound="fp64", achieved=ach, peak=1.25, unit="TFLOP/s", frac=ach / 1.25,
                   peak_source="nominal GB300 float64 rate (no measured figure)",
                   work=f"{solve['iters']} CG iterations x (2 x {solve['nnz']} nnz + block products), block factors")
        return out
    out.update(bound="fp64", achieved=None, peak=1.25, unit="TFLOP/s", frac=None,
               peak_source="nominal GB300 float64 rate (no measured figure)")
    return out


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # a bounded sample per step: the crop shrinks (same source density) so
    # that warmup + steps oracle iterations stay near two and a half minutes
    # (about 2.3 s per iteration on the 512 x 512 crop)
    n = args.warmup + args.steps
    side = int(min(SAMPLE_SIDE, max(128, SAMPLE_SIDE * math.sqrt(150.0 / (2.3 * max(n, 1))))) // 16 * 16)
    res = run_oracle(n, side)
    res["times"] = res["times"][args.warmup:]
    value, cpu = oracle_line(res, side)
    t = statistics.mean(res["times"]) * (1024 * 1024) / (side * side)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": dict(workload_config(), precision="f64 CPU oracle"),
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


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
    args = ap.parse_args()
    if args.oracle_worker:
        oracle_worker(args.oracle_worker, args.oracle_side)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    gpu_arm(args)


if __name__ == "__main__":
    main()
