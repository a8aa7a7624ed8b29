"""Benchmark: batched SVGD full-waveform inversion on one GB300.

One step = one SVGD iteration of the batched FWI workload (120 x 300 grid at
10 m, 20 sources, 200 receivers, 2000 steps at 1 ms, 600 particles):
fwi_gradient for every particle and source (forward + adjoint + imaging in
one persistent cluster launch) followed by svgd_step (tcgen05 Gram, FP64
distances, median bandwidth, fused update with the prior's bound reset).

Prints one JSON line. value = particle-gradients/s over the whole job; the
line also carries cell-update rates, the plain per-step loop's rate on the
same GPU, the roofline of the dominant kernel, the end-to-end rate with host
buffers, the FP64 oracle timed on the host cores, and the SM clocks sampled
during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) the particles are split across the ranks: every rank
holds 600 particles (its own seed) and computes their gradients alone; the
SVGD update couples the whole ensemble of 600 N particles, so each iteration
all-gathers the particles and gradients (NCCL) and every rank applies the
update to the whole ensemble (paper_2310_13325_gb300.sharded). value sums the
ranks' particles over the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "FWI particle-gradients/s (batched SVGD iteration)"
UNIT = "particle-gradients/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cfg3")
    ap.add_argument("--particles", type=int, default=0)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--svgd-kernel", default="rbf", choices=["rbf", "diag"],
                    help="RBF kernel, or the diagonal matrix-valued kernel with Q the "
                         "inverse particle variance")
    ap.add_argument("--svgd-space", default="model", choices=["model", "unconstrained"],
                    help="update the particles with the bound reset, or in the logit-"
                         "transformed space")
    ap.add_argument("--minibatch", type=int, default=0,
                    help="ssvgd workload: gradients from this many uniformly drawn "
                         "sources per step (0 = all), scaled by S / minibatch")
    ap.add_argument("--advi-rank", type=int, default=0,
                    help="ADVI workload: covariance diag + B B^T with B of this rank "
                         "(0 = mean field)")
    ap.add_argument("--advi-rule", default="adam", choices=["sgd", "adagrad", "adadelta", "adam"],
                    help="ascent rule of the ADVI workload")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-fill", action="store_true",
                    help="no second launch on the SMs the batched launch leaves idle")
    ap.add_argument("--plan", default="",
                    help="force the wave launch shape Q,V,T,coeff (cluster CTAs, rows per "
                         "thread, threads, 1 = coefficients in shared / 2 = in global "
                         "memory); profiling cases only")
    ap.add_argument("--nt", type=int, default=0,
                    help="override the number of time steps (profiling cases only)")
    ap.add_argument("--tomo-method", default="svgd", choices=["svgd", "ssvgd", "advi"],
                    help="update of the tomography workload")
    ap.add_argument("--workload", default="svgd",
                    choices=["svgd", "ssvgd", "advi", "tomo", "update"],
                    help="svgd: the batched SVGD step (default); ssvgd / advi: the "
                         "240x600, 40-source shape with the stochastic-SVGD or "
                         "mean-field ADVI update; tomo: the travel-time tomography "
                         "SVGD iteration; update: svgd_step / ssvgd_step alone on "
                         "--particles x --dim random particles")
    ap.add_argument("--dim", type=int, default=36000,
                    help="coordinates per particle of the update workload")
    ap.add_argument("--stochastic", action="store_true",
                    help="update workload: ssvgd_step with injected noise")
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="collective backend of multi-rank runs (gloo: several ranks "
                         "sharing one GPU, gathering through host memory)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_name(cfg, P):
    return ("batched SVGD FWI %dx%d grid dx %g m, %d src, %d rec, %d steps dt %g ms, "
            "%d particles" % (cfg.nz, cfg.nx, cfg.dx, cfg.nsrc, cfg.nrec, cfg.nt,
                              cfg.dt * 1e3, P))


def cell_updates_per_particle(cfg):
    # algorithmic work: forward + adjoint cell updates over the padded grid
    return 2.0 * cfg.nsrc * cfg.nt * cfg.NZ * cfg.NX


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons (read only)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[3 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def build_problem(cfg, P, rank, dev, vg, torch):
    """Synthetic layered model, prior box, particles and observed data. The
    observed traces come from the product's own forward modelling of the true
    model plus seeded noise at the paper's level (Sec. 4.2)."""
    geo = synth.geometry(cfg)
    v_true = synth.true_model(cfg, seed=0)
    lo, hi = synth.prior_bounds(cfg, v_true)
    X0 = synth.particles_from_prior(lo, hi, P, seed=2 + 1000 * rank)
    fwi = vg.Fwi.from_config(cfg, geo)
    clean = fwi.forward(torch.tensor(v_true, dtype=torch.float32, device=dev)[None])[0]
    clean_h = clean.cpu().numpy()
    sigma = synth.sigma_from_traces(clean_h, cfg.sigma_rule)
    dobs = clean_h + sigma * synth.unit_noise(clean_h.shape, seed=1)
    return geo, fwi, X0.astype(np.float32), dobs.astype(np.float32), float(sigma), lo, hi


def run_ours(args, cfg, P, torch, ws_, rank, local):
    import paper_2310_13325_gb300 as vg
    from paper_2310_13325_gb300 import build as vbuild
    from paper_2310_13325_gb300 import sharded
    vbuild.build()
    # one GPU per rank; ranks beyond the visible GPUs (gloo runs that share a
    # GPU) wrap around
    gpu = local % max(1, torch.cuda.device_count())
    dev = torch.device("cuda:%d" % gpu)
    torch.cuda.set_device(dev)
    prec = {"fp32": vg.FWI_FP32, "bf16": vg.FWI_CKPT_BF16, "fp16": vg.FWI_CKPT_FP16}[args.precision]
    gram = vg.VIP_GRAM_BF16X3 if args.precision == "fp32" else vg.VIP_GRAM_BF16
    geo, fwi, X0, dobs_h, sigma, lo, hi = build_problem(cfg, P, rank, dev, vg, torch)
    fwi.set_autotune(not args.no_autotune)
    fwi.set_fill(not args.no_fill)
    if args.plan:
        q, v, t, coeff = (int(x) for x in args.plan.split(","))
        fwi.set_plan(q, v, t, 0, coeff=coeff)
    X = torch.tensor(X0, device=dev)
    dobs = torch.tensor(dobs_h, device=dev)
    lo_t = torch.tensor(lo.reshape(-1), dtype=torch.float32, device=dev)
    hi_t = torch.tensor(hi.reshape(-1), dtype=torch.float32, device=dev)
    misfit = torch.empty(P, dtype=torch.float64, device=dev)
    grad = torch.empty((P, cfg.nz, cfg.nx), dtype=torch.float32, device=dev)
    # the update sees the whole ensemble: P particles on each of the ws_ ranks
    ws = torch.empty(vg.svgd_workspace_size(P * ws_, cfg.d, gram, False), dtype=torch.uint8,
                     device=dev)
    h2 = torch.empty(1, dtype=torch.float64, device=dev)
    qv = torch.empty(cfg.d, dtype=torch.float32, device=dev)
    diag = args.svgd_kernel == "diag"
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    eps_box = {}

    def step():
        fwi.gradient(X, dobs, sigma, precision=prec, misfit=misfit, grad=grad)
        if "eps" not in eps_box:
            # step size: the first update moves the fastest coordinate ~20 m/s
            # (of the whole ensemble: every rank must apply the same update)
            g = grad.abs().max().reshape(1).double()
            if ws_ > 1:
                if args.dist_backend == "gloo":
                    g = g.cpu()
                torch.distributed.all_reduce(g, op=torch.distributed.ReduceOp.MAX)
            eps_box["eps"] = 20.0 / max(g.item(), 1e-30)
        svgd_update()

    uncon = args.svgd_space == "unconstrained"
    if uncon:
        # the transform is undefined on the bounds themselves: prior draws that
        # rounded onto a bound in FP32 start just inside it
        pad = 1e-4 * (hi_t - lo_t)
        X.copy_(torch.minimum(torch.maximum(X, lo_t + pad), hi_t - pad))
    theta = vg.to_unconstrained(X, lo_t, hi_t) if uncon else None
    gth = torch.empty_like(X) if uncon else None

    def update_model_space(Xf, Gf):
        q = vg.svgd_inverse_variance(Xf) if diag else None
        vg.svgd_step(Xf, Gf, eps_box["eps"], lo=lo_t, hi=hi_t, gram_precision=gram, ws=ws,
                     h2_used=h2, gscale=-1.0, q=q)

    def update_unconstrained(Xf, Gf):
        th = vg.to_unconstrained(Xf, lo_t, hi_t)
        gt = vg.unconstrained_gradient(th, Gf, lo_t, hi_t, gscale=-1.0)
        if "eps_t" not in eps_box:
            eps_box["eps_t"] = 0.1 / max(gt.abs().max().item(), 1e-30)
        q = vg.svgd_inverse_variance(th) if diag else None
        vg.svgd_step(th, gt, eps_box["eps_t"], gram_precision=gram, ws=ws, h2_used=h2, q=q)
        vg.to_model(th, lo_t, hi_t, out=Xf)

    def svgd_update():
        if ws_ > 1:
            # particles split across ranks: one all-gather, the update of the
            # whole ensemble on every rank, each keeps its rows
            sharded.sharded_update(X, grad.reshape(P, -1),
                                   update_unconstrained if uncon else update_model_space)
            return
        if not uncon:
            q = vg.svgd_inverse_variance(X, out=qv) if diag else None
            vg.svgd_step(X, grad.reshape(P, -1), eps_box["eps"], lo=lo_t, hi=hi_t,
                         gram_precision=gram, ws=ws, h2_used=h2, gscale=-1.0, q=q)
            return
        # strategy 2 of the uniform prior: the particles live in theta = T(m)
        vg.unconstrained_gradient(theta, grad.reshape(P, -1), lo_t, hi_t, gscale=-1.0, out=gth)
        if "eps_t" not in eps_box:
            eps_box["eps_t"] = 0.1 / max(gth.abs().max().item(), 1e-30)
        q = vg.svgd_inverse_variance(theta, out=qv) if diag else None
        vg.svgd_step(theta, gth, eps_box["eps_t"], gram_precision=gram, ws=ws, h2_used=h2, q=q)
        vg.to_model(theta, lo_t, hi_t, out=X)

    # warm-up (includes the autotuner's timed trials on the first call)
    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    assert fwi.last_status() == 0, "stability bound violated by a particle"

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(gpu)
    if ws_ > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.fill_(1)                      # evict L2 between timed steps
        e0, e1, e2 = ev[k]
        e0.record(stream)
        fwi.gradient(X, dobs, sigma, precision=prec, misfit=misfit, grad=grad)
        e1.record(stream)
        svgd_update()
        e2.record(stream)
    torch.cuda.synchronize()
    if ws_ > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    fwd_ms = [a.elapsed_time(b) for a, b, c in ev]
    svgd_ms = [b.elapsed_time(c) for a, b, c in ev]
    step_ms = [f + s for f, s in zip(fwd_ms, svgd_ms)]
    t_step = float(np.mean(step_ms))
    t_fwi = float(np.mean(fwd_ms))
    t_svgd = float(np.mean(svgd_ms))
    assert torch.isfinite(X).all().item() and torch.isfinite(misfit).all().item()

    plan = fwi.query_plan(P, prec)
    plan["fill"] = fwi.query_fill(P, prec)
    out = {"t_step_ms": t_step, "t_fwi_ms": t_fwi, "t_svgd_ms": t_svgd, "clocks": clocks,
           "plan": plan, "misfit_mean": float(misfit.mean().item()),
           "eps": eps_box["eps"], "h2": float(h2.item())}

    # end to end through the public API with host buffers: pinned inputs in,
    # updated particles and misfits out, every step
    if not args.no_e2e:
        Xh = torch.tensor(X0).pin_memory()
        Dh = torch.tensor(dobs_h).pin_memory()
        Xo = torch.empty_like(Xh).pin_memory()
        Jo = torch.empty(P, dtype=torch.float64).pin_memory()
        ke = max(2, args.steps // 2)
        e_ms = []
        for k in range(ke + 1):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            X.copy_(Xh, non_blocking=True)
            dobs.copy_(Dh, non_blocking=True)
            step()
            Xo.copy_(X, non_blocking=True)
            Jo.copy_(misfit, non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            if k > 0:                       # first pass re-warms the copies
                e_ms.append(a.elapsed_time(b))
        out["e2e_ms"] = float(np.mean(e_ms))
        out["h2d_bytes"] = Xh.numel() * 4 + Dh.numel() * 4
        out["d2h_bytes"] = Xo.numel() * 4 + Jo.numel() * 8

    # the plain per-step GPU loop on a sample (1 particle, 2 sources)
    if not args.no_plain and rank == 0:
        out["plain_particle_gradients_per_s"] = plain_rate(cfg, X[:1], dobs, sigma, vg, torch)
    return out


def plain_rate(cfg, v1, dobs, sigma, vg, torch):
    """Particle-gradients/s of the plain per-step FP32 loop (one launch per time
    step, wavefields in global memory), timed on one particle and two of the
    sources (the first and the middle one) and scaled to all sources."""
    stream = torch.cuda.current_stream()
    sub = cfg.with_(nsrc=2)
    geo2 = synth.geometry(cfg)
    geo2 = dict(geo2, src_iz=geo2["src_iz"][[0, cfg.nsrc // 2]],
                src_ix=geo2["src_ix"][[0, cfg.nsrc // 2]])
    fp = vg.Fwi.from_config(sub, geo2)
    fp.set_mode(vg.FWI_MODE_PLAIN, 1)
    d2 = dobs[[0, cfg.nsrc // 2]].contiguous()
    v1 = v1.clone()
    fp.gradient(v1, d2, sigma)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fp.gradient(v1, d2, sigma)
    b.record(stream)
    torch.cuda.synchronize()
    t_pair = a.elapsed_time(b) / 2.0          # ms per (particle, source)
    fp.close()
    return 1e3 / (t_pair * cfg.nsrc)


# Kernels one svgd_step enqueues (three-piece BF16 Gram, tensor-core update):
# centre, norms, gram_tc, d2_finish, median_init, 8 x median_hist (each radix
# pass selects its digit in its last block), bandwidth, kbar, split_a,
# split_b, rcoef, update_tc, poison.
SVGD_STEP_LAUNCHES = 20


def fwi_gradient_launches(plan, nsrc):
    """The persistent wave kernel (and its fill launch on the idle SMs, when
    there is one), the per-item gradient merge when several work items share a
    particle, and the misfit reduction."""
    fill = 1 if (plan.get("fill") or {}).get("clusters") else 0
    return 1 + fill + (nsrc // plan["sources_per_item"] > 1) + 1


# FP32 lane operations (FADD, FMUL, FFMA: one per lane, packed f32x2 counted
# per lane) of one cell update in the wave kernel's cell loop: horizontal
# neighbour sums 4, the Laplacian bracket 16, the taper update 5; the adjoint
# adds the imaging accumulation (1). Forward and adjoint sweeps alternate, so
# a cell update of the benchmark costs 25.5 on average.
LANE_OPS_PER_CELL_UPDATE = 25.5


def profile_figures():
    """Figures of the committed ncu capture of the wave kernel
    (profiles/wave_traffic.txt): DRAM bytes per cell update and issue-active
    percentage, or None for each when the kernel source has changed since."""
    import hashlib
    try:
        kv = dict(line.strip().split("=", 1) for line in
                  open(os.path.join(ROOT, "profiles", "wave_traffic.txt"))
                  if "=" in line and not line.startswith("#"))
        src = open(os.path.join(ROOT, "paper_2310_13325_gb300", "csrc", "wave.cuh"), "rb").read()
        if hashlib.sha256(src).hexdigest() != kv["wave_cuh_sha256"]:
            return None, None
        issue = float(kv["issue_active_pct"]) if "issue_active_pct" in kv else None
        return float(kv["bytes_per_cell_update"]), issue
    except (OSError, KeyError, ValueError):
        return None, None


def wave_roofline(cell_updates, t_ms, hbm, hbm_src, peaks):
    """Roofline of the dominant kernel (the persistent wave kernel of
    fwi_gradient, 99.9 % of the step's device time). It keeps the wavefields in
    shared memory, so DRAM carries only the stored snapshots; what bounds it is
    instruction issue on the FP32 pipe. Reported against the FP32 lane peak
    (152 SMs x 128 lanes x the maximum SM clock), with the streaming count of
    a stencil that reads its fields from DRAM (16 B per cell update) and the
    measured DRAM traffic against the HBM peak beside it."""
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0)) if peaks else 2070.0
    lane_peak = 152 * 128 * sm_mhz * 1e6 / 1e12               # T lane-op/s
    achieved = LANE_OPS_PER_CELL_UPDATE * cell_updates / (t_ms * 1e-3) / 1e12
    bpc, issue = profile_figures()
    traffic = bpc * cell_updates if bpc else None
    equiv = 16.0 * cell_updates / (t_ms * 1e-3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": lane_peak,
            "unit": "TOP/s (FP32 lane operations)", "frac": achieved / lane_peak,
            "traffic": traffic, "kernel": "wave_cluster_kernel (fwi_gradient)",
            "lane_ops_per_cell_update": LANE_OPS_PER_CELL_UPDATE,
            "peak_source": "152 SMs x 128 FP32 lanes x %.0f MHz (maximum SM clock)" % sm_mhz,
            "issue_active_pct": issue,
            "hbm": {"peak": hbm, "peak_source": hbm_src + " hbm_gbs", "unit": "GB/s",
                    "streaming_equivalent": equiv, "streaming_equivalent_frac": equiv / hbm,
                    "dram": traffic / (t_ms * 1e-3) / 1e9 if traffic else None,
                    "dram_frac": traffic / (t_ms * 1e-3) / 1e9 / hbm if traffic else None,
                    "note": "streaming_equivalent counts 16 B per cell update "
                            "(read a^n, a^{n-1}, w; write a^{n+1}) although the fields stay "
                            "on chip; dram is the ncu-measured traffic (stored snapshots) "
                            "scaled by cell updates"},
            "note": "time = CUDA events around fwi_gradient on its stream (the wave "
                    "kernel, the per-item gradient merge and the misfit reduction)"}


def oracle_pair_seconds(cfg, src=0):
    """Seconds the FP64 oracle, as it stands, takes for one (particle, source)
    forward + adjoint + imaging at the full grid and step count."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import fwi as ofwi
    geo = synth.geometry(cfg)
    g = ofwi.Geom.from_config(cfg, geo)
    v_true = synth.true_model(cfg)
    lo, hi = synth.prior_bounds(cfg, v_true)
    v = synth.particles_from_prior(lo, hi, 1, seed=2)[0].reshape(cfg.nz, cfg.nx)
    dobs0 = np.zeros((g.nrec, g.nt))
    t0 = time.perf_counter()
    ofwi.pair_gradient(v, g, src, lambda tr: tr - dobs0)
    return time.perf_counter() - t0


def _oracle_pair_job(job):
    cfg, src = job
    return oracle_pair_seconds(cfg, src)


def oracle_all_cores(cfg):
    """One (particle, source) pair per host core at once, each in its own
    spawned single-threaded process: (pairs per second, cores, slowest pair s).
    The rate counts the pairs over the slowest pair's own time (process
    start-up excluded)."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        times = pool.map(_oracle_pair_job, [(cfg, k % cfg.nsrc) for k in range(n)])
    return n / max(times), n, max(times)


def cpu_baseline(cfg):
    """The FP64 oracle on the host: one pair single-threaded, then one pair per
    core at once; the reported value is the all-cores rate."""
    t1 = oracle_pair_seconds(cfg)
    rate, n, tmax = oracle_all_cores(cfg)
    return {"value": rate / cfg.nsrc, "unit": UNIT, "cores": n, "kind": "oracle",
            "single_core_value": 1.0 / (t1 * cfg.nsrc),
            "sample": "%d (particle, source) gradients at the full grid and %d steps, one per "
                      "core in spawned single-threaded processes (slowest %.1f s; one alone "
                      "%.1f s), scaled by %d sources per particle"
                      % (n, cfg.nt, tmax, t1, cfg.nsrc)}


def run_reference(args, cfg, P, ws_, rank):
    """Reference arm: the FP64 oracle on the host cores, each step a bounded
    sample of the same workload: one (particle, source) gradient per core at
    once, in spawned single-threaded processes."""
    if rank != 0:
        return
    rates, tmaxes = [], []
    n = 1
    for k in range(args.warmup + args.steps):
        rate, n, tmax = oracle_all_cores(cfg)
        if k >= args.warmup:
            rates.append(rate)
            tmaxes.append(tmax)
    value = float(np.mean(rates)) / cfg.nsrc
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(tmaxes)) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(cfg, P),
                       "sample": "%d particle-source pairs per step, one per core" % n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle",
                             "sample": "per step %d (particle, source) gradients at the full "
                                       "grid, one per core, scaled by %d sources"
                                       % (n, cfg.nsrc)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_other_workload(args, torch):
    """sSVGD or ADVI at the 240 x 600 / 40-source / 3000-step shape. One step:
    ssvgd - fwi_gradient for P particles (default 40, a slice of the
            2000-particle ensemble) and ssvgd_step on all 2000 particles
            (d = 144,000, Cholesky of the 2000 x 2000 kernel, Philox noise);
    advi  - 64 Philox draws, advi_sample, fwi_gradient of the 64 samples,
            advi_step (Adam)."""
    import paper_2310_13325_gb300 as vg
    from paper_2310_13325_gb300 import build as vbuild
    vbuild.build()
    cfg = synth.config("cfg5")
    if args.nt:
        cfg = cfg.with_(nt=args.nt)
    dev = torch.device("cuda:0")
    P = args.particles or (40 if args.workload == "ssvgd" else 64)
    geo, fwi, X0, dobs_h, sigma, lo, hi = build_problem(cfg, max(P, 2000) if args.workload == "ssvgd" else P, 0, dev, vg, torch)
    fwi.set_autotune(not args.no_autotune)
    fwi.set_fill(not args.no_fill)
    prec = {"fp32": vg.FWI_FP32, "bf16": vg.FWI_CKPT_BF16, "fp16": vg.FWI_CKPT_FP16}[args.precision]
    dobs = torch.tensor(dobs_h, device=dev)
    lo_t = torch.tensor(lo.reshape(-1), dtype=torch.float32, device=dev)
    hi_t = torch.tensor(hi.reshape(-1), dtype=torch.float32, device=dev)
    ev = []
    if args.workload == "ssvgd":
        n = X0.shape[0]
        X = torch.tensor(X0, device=dev)
        G = torch.zeros_like(X)
        ws = torch.empty(vg.svgd_workspace_size(n, cfg.d, vg.VIP_GRAM_BF16X3, True),
                         dtype=torch.uint8, device=dev)
        it = [0]

        nbatch = min(args.minibatch, cfg.nsrc) if args.minibatch else cfg.nsrc
        draw = np.random.default_rng(11)

        def step(rec=None):
            sl = X[:P]
            srcs = (np.sort(draw.choice(cfg.nsrc, nbatch, replace=False))
                    if nbatch < cfg.nsrc else None)
            _, g = fwi.gradient(sl, dobs, sigma, precision=prec, sources=srcs)
            G[:P].copy_(g.reshape(P, -1))
            if rec: rec[1].record()
            it[0] += 1
            q = vg.svgd_inverse_variance(X) if args.svgd_kernel == "diag" else None
            # the minibatch sum times S / nb estimates the full-data gradient
            vg.ssvgd_step(X, G, 1e-3, seed=3, it=it[0], lo=lo_t, hi=hi_t, ws=ws,
                          gscale=-cfg.nsrc / nbatch, q=q)
    else:
        d = cfg.d
        mu = torch.tensor(((lo + hi) / 2).reshape(-1), dtype=torch.float32, device=dev)
        a_t, b_t = lo_t - 1.0, hi_t + 1.0
        mu = torch.log((mu - a_t) / (b_t - mu))
        om = torch.full((d,), -3.0, device=dev)
        st = torch.zeros((4, d), device=dev)
        it = [0]

        rank = args.advi_rank
        if rank:
            Bl = torch.zeros((d, rank), device=dev)
            st_lr = torch.zeros(4 * d + 2 * d * rank, device=dev)
            work = torch.empty(2 * rank * rank, dtype=torch.float64, device=dev)

        def step(rec=None):
            it[0] += 1
            eta = vg.philox_normal(P, d, seed=5, it=it[0], device=dev)
            if rank:
                epsl = vg.philox_normal(P, rank, seed=6, it=it[0], device=dev)
                m = vg.advi_lowrank_sample(mu, om, Bl, eta, epsl, a_t, b_t)
            else:
                m = vg.advi_sample(mu, om, eta, a_t, b_t)
            _, g = fwi.gradient(m, dobs, sigma, precision=prec)
            if rec: rec[1].record()
            if rank:
                vg.advi_lowrank_step(mu, om, Bl, st_lr, it[0], eta, epsl, g.reshape(P, -1), 0.01,
                                     a_t, b_t, gscale=-1.0, work=work)
                return
            rule = {"sgd": vg.ASCENT_SGD, "adagrad": vg.ASCENT_ADAGRAD,
                    "adadelta": vg.ASCENT_ADADELTA, "adam": vg.ASCENT_ADAM}[args.advi_rule]
            lr = 1.0 if rule == vg.ASCENT_ADADELTA else 0.01
            vg.advi_step_opt(mu, om, st, it[0], eta, g.reshape(P, -1), lr, rule, a_t, b_t,
                             gscale=-1.0)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        step(e)
        e[2].record()
        ev.append(e)
    torch.cuda.synchronize()
    t_step = float(np.mean([a.elapsed_time(c) for a, b, c in ev]))
    t_fwi = float(np.mean([a.elapsed_time(b) for a, b, c in ev]))
    t_upd = float(np.mean([b.elapsed_time(c) for a, b, c in ev]))
    cu = cell_updates_per_particle(cfg)
    nsrc_used = cfg.nsrc
    if args.workload == "ssvgd" and args.minibatch:
        nsrc_used = min(args.minibatch, cfg.nsrc)
        cu = cu * nsrc_used / cfg.nsrc      # a minibatch gradient covers nsrc_used sources
    line = {"metric": "FWI particle-gradients/s (%s step, 240x600 shape)" % args.workload,
            "value": P / (t_fwi * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%s 240x600 grid dx 10 m, 40 src, 400 rec, %d steps dt 0.8 ms, "
                                   "%d gradients per step" % (args.workload, cfg.nt, P),
                       "precision": args.precision, "sources_per_gradient": nsrc_used,
                       "plan": dict(fwi.query_plan(P, prec), fill=fwi.query_fill(P, prec))},
            "gcell_updates_per_s": cu * P / (t_fwi * 1e-3) / 1e9,
            "fwi_ms_per_step": t_fwi, "update_ms_per_step": t_upd,
            "update": ("ssvgd_step n=2000 d=144000, %s kernel" % args.svgd_kernel
                       if args.workload == "ssvgd"
                       else ("advi_lowrank_step S=64 d=144000 rank %d" % args.advi_rank
                             if args.advi_rank else
                             "advi_step S=64 d=144000, %s" % args.advi_rule))}
    if args.workload == "ssvgd":
        line["iteration_s_for_2000_particles"] = (2000.0 / P) * t_fwi * 1e-3 + t_upd * 1e-3
    if not args.no_plain:
        # the same gradients through the plain per-step FP32 loop
        pr = plain_rate(cfg, torch.tensor(X0[:1], device=dev), dobs, sigma, vg, torch)
        line["plain_particle_gradients_per_s"] = pr
        line["batched_over_plain"] = line["value"] / pr
    print(json.dumps(line))


def _tomo_oracle_job(job):
    """Seconds of the FP64 oracle for one whole tomography particle gradient."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import tomo as otomo
    cfg, sta, dobs, sig, x = job
    t0 = time.perf_counter()
    otomo.misfit_gradient(x.reshape(cfg.ny, cfg.nx), cfg.h, sta, dobs, sig)
    return time.perf_counter() - t0


def tomo_cpu_baseline(cfg, sta, dobs, sig, X):
    """The FP64 oracle as it stands on whole particles of the tomography
    workload (every source, every ray): one particle alone, then one particle
    per host core at once in spawned single-threaded processes."""
    import multiprocessing as mp
    t1 = _tomo_oracle_job((cfg, sta, dobs, sig, X[0]))
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        times = pool.map(_tomo_oracle_job,
                         [(cfg, sta, dobs, sig, X[k % len(X)]) for k in range(n)])
    return {"value": n / max(times), "unit": "particle-gradients/s", "cores": n,
            "kind": "oracle", "single_core_value": 1.0 / t1,
            "sample": "%d whole particle gradients (%d sources, %d rays each), one per core "
                      "in spawned single-threaded processes (slowest %.1f s; one alone %.1f s)"
                      % (n, cfg.n_stations - 1, cfg.n_pairs, max(times), t1)}


def run_tomo(args, torch):
    """Travel-time tomography iteration at the Sec. 4.1 shape (40 x 37 nodes of
    0.33 degrees, 61 stations, 1830 station pairs, uniform prior handled in the
    unconstrained space), with the paper's three methods:
      svgd  - 500 particles: ray gradients, transform to theta, svgd_step, back;
      ssvgd - 20 particles: the same with ssvgd_step (Philox noise);
      advi  - 64 draws of the mean-field Gaussian in theta: advi_sample, ray
              gradients, advi_step_opt (Adam)."""
    import synth.tomo as st
    import paper_2310_13325_gb300 as vg
    from paper_2310_13325_gb300 import build as vbuild
    vbuild.build()
    method = args.tomo_method
    cfg = st.tomo_config("tomo_uk")
    P = args.particles or {"svgd": cfg.n_particles, "ssvgd": 20, "advi": 64}[method]
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    sta = st.stations(cfg)
    tm = vg.Tomo.from_config(cfg, sta)
    sig_h = st.pair_sigma(cfg, sta).astype(np.float32)
    sig = torch.tensor(sig_h, device=dev)
    v_true = torch.tensor(st.true_group_velocity(cfg).astype(np.float32), device=dev)
    clean = tm.traveltimes(v_true.reshape(1, -1))[0]
    dobs = clean + sig * torch.tensor(st.unit_noise(tm.n_pairs).astype(np.float32), device=dev)
    lo, hi = st.prior_bounds(cfg)
    lo_t = torch.tensor(lo.reshape(-1), dtype=torch.float32, device=dev)
    hi_t = torch.tensor(hi.reshape(-1), dtype=torch.float32, device=dev)
    # the transform is undefined on the bounds: draws start just inside them
    pad = 1e-4 * (cfg.vmax - cfg.vmin)
    X0 = np.clip(st.particles_from_prior(cfg, P), cfg.vmin + pad,
                 cfg.vmax - pad).astype(np.float32)
    X = torch.tensor(X0, device=dev)
    theta = vg.to_unconstrained(X, lo_t, hi_t)
    gth = torch.empty_like(X)
    misfit = torch.empty(P, dtype=torch.float64, device=dev)
    grad = torch.empty((P, cfg.ny, cfg.nx), device=dev)
    gram = vg.VIP_GRAM_BF16X3
    ws = (torch.empty(vg.svgd_workspace_size(P, cfg.d, gram, method == "ssvgd"),
                      dtype=torch.uint8, device=dev) if method != "advi" else None)
    h2 = torch.empty(1, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    mu = torch.zeros(cfg.d, device=dev)              # standard Gaussian start in theta
    om = torch.zeros(cfg.d, device=dev)
    adam = torch.zeros((4, cfg.d), device=dev)
    eta = torch.empty((P, cfg.d), device=dev)
    box = {"it": 0}
    S = cfg.n_stations - 1
    nb = min(args.minibatch, S) if args.minibatch else S
    draw = np.random.default_rng(11)

    def gradient():
        # a source minibatch sums nb of the S source stations' pairs; S / nb
        # times it estimates the full-data gradient (Sec. 3 after Eq. 22)
        srcs = np.sort(draw.choice(S, nb, replace=False)) if nb < S else None
        tm.gradient(X, dobs, sig, misfit=misfit, grad=grad, sources=srcs)

    def prepare():
        if method == "advi":
            box["it"] += 1
            vg.philox_normal(P, cfg.d, seed=5, it=box["it"], out=eta, device=dev)
            vg.advi_sample(mu, om, eta, lo_t, hi_t, out=X)

    def update():
        if method == "advi":
            vg.advi_step_opt(mu, om, adam, box["it"], eta, grad.reshape(P, -1), 0.01,
                             vg.ASCENT_ADAM, lo_t, hi_t, gscale=-S / nb)
            return
        vg.unconstrained_gradient(theta, grad.reshape(P, -1), lo_t, hi_t, gscale=-S / nb,
                                  out=gth)
        if "eps" not in box:
            box["eps"] = 0.05 / max(gth.abs().max().item(), 1e-30)
        if method == "ssvgd":
            box["it"] += 1
            vg.ssvgd_step(theta, gth, box["eps"], seed=3, it=box["it"], gram_precision=gram,
                          ws=ws, h2_used=h2)
        else:
            vg.svgd_step(theta, gth, box["eps"], gram_precision=gram, ws=ws, h2_used=h2)
        vg.to_model(theta, lo_t, hi_t, out=X)

    def step():
        prepare()
        gradient()
        update()

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    assert tm.last_status() == 0
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    ev = []
    for _ in range(args.steps):
        flush.fill_(1)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        prepare()
        gradient()
        e[1].record(stream)
        update()
        e[2].record(stream)
        ev.append(e)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    assert tm.last_status() == 0 and torch.isfinite(X).all().item()
    t_step = float(np.mean([a.elapsed_time(c) for a, b, c in ev]))
    t_grad = float(np.mean([a.elapsed_time(b) for a, b, c in ev]))
    t_upd = float(np.mean([b.elapsed_time(c) for a, b, c in ev]))

    # end to end with host buffers: the method's state and the data in, the
    # state and the misfits out
    state = [mu, om] if method == "advi" else [X]
    hin = [t.cpu().pin_memory() for t in state] + [dobs.cpu().pin_memory()]
    hout = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in state]
    Jo = torch.empty(P, dtype=torch.float64).pin_memory()
    e_ms = []
    for k in range(max(2, args.steps // 2) + 1):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for dst, src in zip(state + [dobs], hin):
            dst.copy_(src, non_blocking=True)
        if method != "advi":
            vg.to_unconstrained(X, lo_t, hi_t, out=theta)
        step()
        for dst, src in zip(hout, state):
            dst.copy_(src, non_blocking=True)
        Jo.copy_(misfit, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if k > 0:
            e_ms.append(a.elapsed_time(b))
    e2e = float(np.mean(e_ms))
    name = {"svgd": "SVGD", "ssvgd": "sSVGD", "advi": "ADVI (Adam)"}[method]
    line = {"metric": "tomography particle-gradients/s (%s iteration)" % name,
            "value": P / (t_step * 1e-3), "unit": "particle-gradients/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "%s travel-time tomography, 40x37 nodes of 0.33 deg, "
                                   "%d stations, %d pairs, %d %s, unconstrained space"
                                   % (name, cfg.n_stations, cfg.n_pairs, P,
                                      "samples" if method == "advi" else "particles"),
                       "sources_per_gradient": nb,
                       "l2": "flushed between timed steps (256 MB write)"},
            "gradient_ms_per_step": t_grad, "update_ms_per_step": t_upd,
            "eikonal_solves_per_s": P * nb / (t_grad * 1e-3),
            "clocks": clocks,
            "e2e": {"value": P / (e2e * 1e-3), "unit": "particle-gradients/s",
                    "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in hin),
                    "d2h_bytes_per_step": (sum(t.numel() * t.element_size() for t in hout)
                                           + Jo.numel() * 8)}}
    if method == "svgd":
        # tomo_kernel, tomo_misfit_kernel, the transform pair and svgd_step
        line["gpu_launches"] = (2 + 2 + SVGD_STEP_LAUNCHES) * args.steps
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = tomo_cpu_baseline(cfg, sta, dobs.cpu().double().numpy(),
                                                 sig_h.astype(np.float64), X0.astype(np.float64))
    print(json.dumps(line))


def run_update(args, torch):
    """svgd_step or ssvgd_step (injected unit-normal noise) alone on seeded
    standard-normal particles and gradients [--particles, --dim], three-piece
    BF16 Gram and the tensor-core update: milliseconds per call."""
    import paper_2310_13325_gb300 as vg
    from paper_2310_13325_gb300 import build as vbuild
    vbuild.build()
    n, d = args.particles or 600, args.dim
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(7)
    X0 = torch.tensor(rng.standard_normal((n, d)).astype(np.float32), device=dev)
    G = torch.tensor(rng.standard_normal((n, d)).astype(np.float32), device=dev)
    xi = torch.tensor(rng.standard_normal((n, d)).astype(np.float32), device=dev)
    gram = vg.VIP_GRAM_BF16X3
    ws = torch.empty(vg.svgd_workspace_size(n, d, gram, args.stochastic), dtype=torch.uint8,
                     device=dev)
    X = X0.clone()

    def call():
        X.copy_(X0)
        if args.stochastic:
            vg.ssvgd_step(X, G, 1e-3, seed=3, it=1, xi=xi, gram_precision=gram, ws=ws)
        else:
            vg.svgd_step(X, G, 1e-3, gram_precision=gram, ws=ws)

    for _ in range(max(args.warmup, 3)):
        call()
    torch.cuda.synchronize()
    ev = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        call()
        b.record()
        ev.append((a, b))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    line = {"metric": "%s time" % ("ssvgd_step" if args.stochastic else "svgd_step"),
            "value": ms, "unit": "ms", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%d particles x %d coordinates, three-piece BF16 "
                                   "Gram, tensor-core update" % (n, d)}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = update_cpu_baseline(n, d, args.stochastic)
    print(json.dumps(line))


def update_cpu_baseline(n, d, stochastic):
    """The FP64 oracle's svgd_step / ssvgd_step as it stands, in this process,
    on a bounded sample: ns = min(n, 150) seeded particles of the same d. Its
    work grows as n^2 d (the pairwise distances, taken row by row, and the
    kernel products), so the time is scaled by (n / ns)^2."""
    from oracle import svgd as osvgd
    ns = min(n, 150)
    rng = np.random.default_rng(7)
    X, G, xi = (rng.standard_normal((ns, d)) for _ in range(3))
    t0 = time.perf_counter()
    if stochastic:
        osvgd.ssvgd_step(X, G, 1e-3, xi)
    else:
        osvgd.svgd_step(X, G, 1e-3)
    dt = time.perf_counter() - t0
    return {"value": dt * 1e3 * (n / ns) ** 2, "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": "one oracle %s on %d x %d particles (%.1f s), scaled by (%d / %d)^2; "
                      "one process (its row loops on one core, K @ G on the BLAS threads)"
                      % ("ssvgd_step" if stochastic else "svgd_step", ns, d, dt, n, ns)}


def reduce_over_ranks(t_ms, e2e_ms, device):
    """Slowest rank's step time and end-to-end time (max over ranks)."""
    import torch
    t = torch.tensor([t_ms, e2e_ms or 0.0], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t[0]), (float(t[1]) or None)


def job_value(particles_per_rank, world, t_max_ms):
    """Whole-job particle-gradients/s: all ranks' particles over the slowest
    rank's step time."""
    return particles_per_rank * world / (t_max_ms * 1e-3)


def main():
    args = parse()
    ws_, rank, local = dist_env()
    cfg = synth.config(args.config)
    if args.nt:
        cfg = cfg.with_(nt=args.nt)
    P = args.particles or cfg.n_particles
    if args.impl == "reference":
        run_reference(args, cfg, P, ws_, rank)
        return
    import torch
    if args.workload == "tomo":
        run_tomo(args, torch)
        return
    if args.workload == "update":
        run_update(args, torch)
        return
    if args.workload != "svgd":
        run_other_workload(args, torch)
        return
    if ws_ > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.distributed.init_process_group(args.dist_backend)
    res = run_ours(args, cfg, P, torch, ws_, rank, local)
    t_max = res["t_step_ms"]
    e2e_max = res.get("e2e_ms")
    if ws_ > 1:
        t_max, e2e_max = reduce_over_ranks(t_max, e2e_max, "cpu" if args.dist_backend == "gloo"
                                           else "cuda:%d" % (local % torch.cuda.device_count()))
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    units = P * ws_
    value = job_value(P, ws_, t_max)
    cu = cell_updates_per_particle(cfg)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm = float(peaks["hbm_gbs"]); src = "measured"
    except Exception:
        hbm = 6800.0; src = "fallback"
    line_roof = wave_roofline(cu * P, res["t_fwi_ms"], hbm, src, peaks)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(cfg, P), "precision": args.precision,
                   "svgd_kernel": args.svgd_kernel, "svgd_space": args.svgd_space,
                   "l2": "flushed between timed steps (256 MB write)",
                   "plan": res["plan"]},
        "gcell_updates_per_s": cu * units / (t_max * 1e-3) / 1e9,
        "fwi_ms_per_iter": res["t_fwi_ms"], "svgd_ms_per_iter": res["t_svgd_ms"],
        "plain_particle_gradients_per_s": res.get("plain_particle_gradients_per_s"),
        "batched_over_plain": (value / ws_ / res["plain_particle_gradients_per_s"]
                               if res.get("plain_particle_gradients_per_s") else None),
        "roofline": line_roof,
        "gpu_launches": (fwi_gradient_launches(res["plan"], cfg.nsrc) + SVGD_STEP_LAUNCHES +
                         (args.svgd_kernel == "diag") +
                         2 * (args.svgd_space == "unconstrained")) * args.steps,
        "clocks": res["clocks"],
    }
    if e2e_max:
        line["e2e"] = {"value": job_value(P, ws_, e2e_max), "unit": UNIT,
                       "h2d_bytes_per_step": res["h2d_bytes"],
                       "d2h_bytes_per_step": res["d2h_bytes"]}
    # the FP64 oracle on the host cores: rank 0 of a single-GPU run only (a
    # multi-GPU run would hold every GPU while it runs)
    if not args.no_cpu_baseline and ws_ == 1:
        line["cpu_baseline"] = cpu_baseline(cfg)
    print(json.dumps(line))
    if ws_ > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
