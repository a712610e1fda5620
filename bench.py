#!/usr/bin/env python3
"""Benchmark of the FMM-compressed single-layer operator on one GB300.

Workload: interior Laplace problem on the unit sphere (6 cube-sphere patches),
degree-3 B-splines on level 5 (7,350 dofs, 98,304 superspace dofs), Chebyshev
6 x 6 points per cluster, admissibility eta = 1.6, one right-hand side.

A step is one application of y = T A T^T x (lift, upward pass, coupling,
downward pass, near field, restriction), the operator applied in every Krylov
iteration.  `value` is dofs x right-hand sides per second of the FP64 operator
over all ranks (each rank runs an independent replica; no data-path
collective).  Beside it: the FP32 operator (error against FP64 stated), the
FP64 CG solve and the mixed-precision iterative-refinement solve to true
relative residual 1e-8, the end-to-end time through ibem_matvec_host with host
buffers, the roofline of the dominant kernel and the oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "laplace-sphere-p3-m5-q6-eta1.6", "p": 3, "m": 5, "q_cheb": 6, "eta": 1.6,
            "nrhs": 1, "geometry": "unit sphere, 6 cube-sphere patches", "kernel": "laplace"}
METRIC = "FMM single-layer matvec DOF*RHS/s (FP64), GMRES/CG solve time to 1e-8 vs plain FP64 GPU"
UNIT = "DOF*RHS/s"
SEED = 170809162
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "coupling_df_kernel_laplace_sphere_p3_m5.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-native", action="store_true", help="skip the native-FP64-coupling comparison")
    ap.add_argument("--no-helmholtz-many", action="store_true", help="skip the many-right-hand-side Helmholtz section")
    ap.add_argument("--helmholtz-many-only", action="store_true", help="run only the many-right-hand-side section")
    ap.add_argument("--helmholtz-many-m", type=int, default=6, help="refinement level of that section (profiling)")
    ap.add_argument("--m", type=int, default=None, help="refinement level override (profiling cases)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner section")
    ap.add_argument("--learned-only", action="store_true", help="run only the learned-preconditioner section")
    ap.add_argument("--cnn-forward-only", action="store_true", help="time only the network's forward pass")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances section")
    ap.add_argument("--batch-only", action="store_true", help="run only the batched-instances section")
    ap.add_argument("--learn-train-m", type=int, default=5, help="level of the training solves")
    ap.add_argument("--learn-m", type=int, default=6, help="level of the compared solves")
    ap.add_argument("--learn-nrhs", type=int, default=2, help="plane waves of the compared solves")
    ap.add_argument("--oracle-worker", type=int, default=0, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------- oracle timing
def oracle_worker(nrows):
    """Runs in a child process with one BLAS thread: times nrows rows of the
    oracle's FMM-mode operator on the benchmark workload; prints one JSON line."""
    import numpy as np
    from oracle import fmm, galerkin, geometry
    t0 = time.perf_counter()
    disc = galerkin.Discretisation(geometry.unit_sphere(), WORKLOAD["p"], WORKLOAD["m"], galerkin.LaplaceKernel())
    op = fmm.FMMOperator(disc, WORKLOAD["q_cheb"], WORKLOAD["eta"])
    setup = time.perf_counter() - t0
    rng = np.random.default_rng(SEED)
    x = rng.normal(size=disc.mesh.n_dofs)
    rows = rng.choice(disc.mesh.n_dofs, size=nrows, replace=False)
    times = []
    for r in rows:
        op._near_blocks.clear()
        t = time.perf_counter()
        op.rows([int(r)], x)
        times.append(time.perf_counter() - t)
    print(json.dumps({"rows": int(nrows), "seconds": sum(times), "setup_s": setup}))


def run_oracle(nrows):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", str(nrows)],
                         capture_output=True, text=True, env=env, cwd=ROOT)
    if out.returncode != 0:
        raise RuntimeError("oracle worker failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def reference_arm(args, rank):
    """The oracle, as it stands, on the host cores: each step computes 2 rows."""
    if rank != 0:
        return
    per_step = 2
    import numpy as np
    from oracle import fmm, galerkin, geometry
    disc = galerkin.Discretisation(geometry.unit_sphere(), WORKLOAD["p"], WORKLOAD["m"], galerkin.LaplaceKernel())
    op = fmm.FMMOperator(disc, WORKLOAD["q_cheb"], WORKLOAD["eta"])
    rng = np.random.default_rng(SEED)
    x = rng.normal(size=disc.mesh.n_dofs)

    def step():
        op._near_blocks.clear()
        op.rows([int(r) for r in rng.choice(disc.mesh.n_dofs, per_step, replace=False)], x)

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t
    value = args.steps * per_step / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, l2="n/a (host)"), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d rows of the FMM-mode operator per step (one BLAS thread)" % per_step},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _profile_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary."""
    try:
        for line in open(PROFILE_SUMMARY):
            if line.startswith("traffic_bytes_per_launch:"):
                return float(line.split(":")[1])
    except OSError:
        pass
    return None


def max_over_ranks(value):
    """The largest of the ranks' values (a time), through the initialised process
    group (NCCL on the GPUs, or gloo on the host); the value itself with one rank."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(value)
    dev = "cuda" if td.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    except OSError:
        return 6800.0, 2070.0, "fallback"


def helmholtz_many_rhs(ibem, stream, world, barrier, args):
    """Exterior Helmholtz, kappa = 4, p = 2, m = 6, q = 8, 64 incident plane waves
    (seeded uniform directions): the FP32 operator with the coupling on the
    tensor cores, its error against the FP64 operator on one right-hand side,
    and the roofline of the tensor-core coupling kernel."""
    import numpy as np
    import torch
    p, m, q, kappa, R = 2, args.helmholtz_many_m, 8, 4.0, 64
    t0 = time.perf_counter()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(p, m, q_cheb=q, eta=1.6, kernel=ibem.IBEM_HELMHOLTZ,
                                                                 kappa=kappa), stream)
    ibem.ibem_assemble(h)
    setup_s = time.perf_counter() - t0
    info = ibem.ibem_get_info(h)
    N = info.ndof
    rng = np.random.default_rng(SEED + 3)
    d = rng.normal(size=(R, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    torch.cuda.synchronize()
    ph = qp.cpu().numpy() @ d.T                                    # [nq, R]
    g = -np.exp(1j * kappa * ph).T                                 # sound-soft data, [R, nq]
    gq = torch.from_numpy(np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))).cuda()
    b = torch.empty((R, N, 2), dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, gq, R, b)
    y = torch.empty_like(b)
    steps = max(3, args.steps // 20)
    with torch.cuda.stream(stream):
        for _ in range(2):
            ibem.ibem_matvec(h, b, y, R, ibem.IBEM_FP32)
    barrier()
    ibem.ibem_profile_enable(h, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(steps):
            ibem.ibem_matvec(h, b, y, R, ibem.IBEM_FP32)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1) / steps
    prof = ibem.ibem_profile_read(h)
    ibem.ibem_profile_enable(h, False)
    coup_ms = prof["ms"]["coupling"] / steps
    phases = {k: v / steps for k, v in prof["ms"].items()}
    # FP64 operator on the first right-hand side (coupling generated on the fly in FP64)
    y64 = torch.empty((1, N, 2), dtype=torch.float64, device="cuda")
    t1 = time.perf_counter()
    ibem.ibem_matvec(h, b[:1].contiguous(), y64, 1, ibem.IBEM_FP64)
    torch.cuda.synchronize()
    fp64_s = time.perf_counter() - t1
    err = float((y[0] - y64[0]).abs().max() / y64[0].abs().max())
    # potential of the 64 densities (the right-hand sides stand in for them) at 200
    # points on the sphere of radius 3 (seeded): one e^{ikr}/r per point, source
    # and chunk of 16 densities, FP64
    npt = 200
    dp = rng.normal(size=(npt, 3))
    pts = torch.from_numpy(3.0 * dp / np.linalg.norm(dp, axis=1)[:, None]).cuda()
    u = torch.empty((R, npt, 2), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        ibem.ibem_potential(h, b, R, pts, u)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(2):
            ibem.ibem_potential(h, b, R, pts, u)
    e1.record(stream)
    torch.cuda.synchronize()
    pot_ms = e0.elapsed_time(e1) / 2
    nsrc = info.n_elements * 64
    # the same potentials with the far field interpolated (forward moments of the
    # 64 densities, per-point tree walk, q^2 kernel values per admissible cluster)
    uf = torch.empty_like(u)
    with torch.cuda.stream(stream):
        nf, nn = ibem.ibem_potential_fmm(h, b, R, pts, uf)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(5):
            ibem.ibem_potential_fmm(h, b, R, pts, uf)
    e1.record(stream)
    torch.cuda.synchronize()
    fmm_ms = e0.elapsed_time(e1) / 5
    fmm_err = float((uf - u).abs().max() / u.abs().max())
    potential = {"points": npt, "densities": R, "sources": nsrc, "ms": pot_ms,
                 "pair_density_evals_per_s": npt * nsrc * R / (pot_ms * 1e-3),
                 "kernel_evals_per_s": npt * nsrc * ((R + 15) // 16) / (pot_ms * 1e-3),
                 "interpolated": {"ms": fmm_ms, "far_terms": nf, "near_terms": nn, "speedup": pot_ms / fmm_ms,
                                  "rel_err_vs_direct": fmm_err}}
    q2 = q * q
    flops = 2.0 * 128 * 128 * 64 * info.n_far                      # real-form GEMM per far block
    peak = 1912.6
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = json.load(f).get("bf16_tflops", peak)
    except OSError:
        pass
    sfu = 3.0 * q2 * q2 * info.n_far                               # rsqrt, sine, cosine per complex entry
    sfu_peak = 152 * 16 * 2070e6
    ibem.ibem_destroy(h)
    return {"workload": "helmholtz-sphere-p2-m%d-q8-k4-R64" % m, "ndof": N, "ndof_super": info.ndof_super,
            "n_near": info.n_near, "n_far": info.n_far, "nrhs": R, "setup_s": setup_s,
            "value": world * N * R / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "coupling_ms": coup_ms,
            "phase_ms": phases,
            "rel_err_vs_fp64_rhs0": err, "fp64_one_rhs_s": fp64_s, "potential": potential,
            "tensor": {"kernel": "mr_coupling_tc_kernel", "achieved_tflops": flops / (coup_ms * 1e-3) / 1e12,
                       "peak_tflops": peak, "frac": flops / (coup_ms * 1e-3) / 1e12 / peak,
                       "sfu_frac": sfu / (coup_ms * 1e-3) / sfu_peak,
                       "note": "K is generated per block on the SFU (rsqrt, sine, cosine); the tensor pipe waits "
                               "for it"}}


def batched_instances(ibem, stream, args):
    """Many uneven problem instances in one application: 24 seeded instances
    (levels 2-4, degrees 1-3, Laplace or Helmholtz with kappa in [2, 8], q 6 or
    8, 1-16 right-hand sides, spheres of radius 0.5-2), the FP32 operator with
    the coupling generated on the fly (no FP64 coupling stored).  The batched,
    graph-captured application is timed against the same instances applied one
    after another through ibem_matvec."""
    import numpy as np
    import torch
    rng = np.random.default_rng(SEED + 7)
    handles, nrhs, dofs = [], [], 0
    t0 = time.perf_counter()
    for _ in range(24):
        kern = int(rng.integers(0, 2))
        p, m, q = int(rng.integers(1, 4)), int(rng.integers(2, 5)), int(rng.choice([6, 8]))
        R = int(rng.integers(1, 17))
        kappa = float(rng.uniform(2.0, 8.0)) if kern else 0.0
        rad = float(rng.uniform(0.5, 2.0))
        h = ibem.ibem_create(ibem.sphere_patches(rad), ibem.make_params(p, m, q_cheb=q, kernel=kern, kappa=kappa,
                                                                        fp64_coupling=ibem.IBEM_COUPLING_NONE), stream)
        ibem.ibem_assemble(h)
        handles.append(h)
        nrhs.append(R)
        dofs += ibem.ibem_get_info(h).ndof * R
    setup_s = time.perf_counter() - t0
    b = ibem.ibem_batch_create(handles, nrhs, stream)
    off = ibem.ibem_batch_offsets(b, len(handles))
    x = torch.from_numpy(rng.normal(size=off[-1])).cuda()
    y = torch.zeros_like(x)
    ys = torch.zeros_like(x)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
        ev0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(reps):
                fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    def one_by_one():
        for i, h in enumerate(handles):
            ibem.ibem_matvec(h, x[off[i]:off[i + 1]], ys[off[i]:off[i + 1]], nrhs[i], ibem.IBEM_FP32)

    batched_ms = timed(lambda: ibem.ibem_batch_matvec(b, x, y))
    single_ms = timed(one_by_one)
    diff = float((y - ys).abs().max() / ys.abs().max())
    info = ibem.ibem_batch_info(b)
    ibem.ibem_batch_destroy(b)
    for h in handles:
        ibem.ibem_destroy(h)
    return {"instances": len(handles), "dof_rhs_per_apply": dofs, "setup_s": setup_s,
            "batched_ms": batched_ms, "one_by_one_ms": single_ms, "speedup": single_ms / batched_ms,
            "value": dofs / (batched_ms * 1e-3), "unit": UNIT, "rel_diff_batched_vs_one_by_one": diff,
            "launches_per_apply": info["launches_per_apply"], "coupling_threads": info["coupling_threads"]}


def cnn_forward_timing(ibem, stream, c):
    """The network's BF16 forward pass (tensor cores) on 96 images of 130 x 130
    (level 7, 16 right-hand sides x 6 patches), CUDA events on the bench stream,
    20 repetitions after 3 warm-up, against the measured HBM bandwidth (the
    convolutions are memory-bound) and the measured BF16 tensor peak."""
    import torch
    B, H = 96, 130
    x = torch.randn((B, 2, H, H), dtype=torch.float32, device="cuda")
    out = torch.empty_like(x)
    with torch.cuda.stream(stream):
        for _ in range(3):
            ibem.ibem_cnn_forward(c, x, out, ibem.IBEM_BF16)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    ev0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(reps):
            ibem.ibem_cnn_forward(c, x, out, ibem.IBEM_BF16)
    ev1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = ev0.elapsed_time(ev1) / reps
    C = 32
    flops = 2.0 * 9 * (2 * C + C * C + C * C + C * 2) * B * H * H
    # algorithmic bytes per pixel: FP32 input (8), packed input written and read
    # (16 + 16), three 32-channel BF16 activations written and read (3 x 128),
    # BF16 output (4)
    nbytes = (8 + 16 + 16 + 3 * 128 + 4) * B * H * H
    hbm, _, src = _peaks()
    bf16_peak = 1912.6
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak = json.load(f).get("bf16_tflops", bf16_peak)
    except OSError:
        pass
    return {"images": B, "size": H, "ms": fwd_ms, "kernels": "conv_tc_kernel (tcgen05) x 4",
            "bound": "hbm", "algorithmic_bytes": nbytes,
            "achieved_gbs": nbytes / (fwd_ms * 1e-3) / 1e9, "peak_gbs": hbm,
            "frac": nbytes / (fwd_ms * 1e-3) / 1e9 / hbm,
            "tflops": flops / (fwd_ms * 1e-3) / 1e12, "bf16_peak_tflops": bf16_peak,
            "tensor_frac": flops / (fwd_ms * 1e-3) / 1e12 / bf16_peak,
            "peak_note": "MEASURED_PEAKS.json (%s)" % src,
            "device_status": ibem.ibem_cnn_device_status(c)}


def learned_preconditioner(ibem, stream, args):
    """Learned right preconditioner, Helmholtz sound-soft scattering on the
    6-patch sphere, p = 2, q = 6, k drawn uniformly from [8, 16] (seeded):
    the network (32 channels) is trained on unit-norm residuals of plain
    block-Jacobi GMRES solves at level args.learn_train_m (three wavenumbers,
    two plane waves each) with the residual-norm objective, then flexible GMRES
    with it is compared with block-Jacobi GMRES at level args.learn_m on
    args.learn_nrhs plane waves, both on the FP64 operator to relative residual
    1e-8.  Also the network's forward pass on 16 right-hand sides' worth of
    130 x 130 images (level 7)."""
    import numpy as np
    import torch
    rng = np.random.default_rng(SEED + 5)
    p, q = 2, 6

    def make(m, k):
        h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(p, m, q_cheb=q, eta=1.6,
                                                                     kernel=ibem.IBEM_HELMHOLTZ, kappa=k), stream)
        ibem.ibem_assemble(h)
        return h

    def plane_rhs(h, k, n):
        info = ibem.ibem_get_info(h)
        d = rng.normal(size=(n, 3))
        d /= np.linalg.norm(d, axis=1)[:, None]
        qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
        ibem.ibem_quad_points(h, qp)
        torch.cuda.synchronize()
        g = -np.exp(1j * k * (qp.cpu().numpy() @ d.T)).T
        gq = torch.from_numpy(np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))).cuda()
        b = torch.empty((n, info.ndof, 2), dtype=torch.float64, device="cuda")
        ibem.ibem_rhs(h, gq, n, b)
        return b

    c = ibem.ibem_cnn_create(32, seed=SEED, stream=stream)
    t0 = time.perf_counter()
    train = []
    for k in rng.uniform(8.0, 16.0, size=3):
        h = make(args.learn_train_m, k)
        info = ibem.ibem_get_info(h)
        b = plane_rhs(h, k, 2)
        r = torch.zeros((2 * 60, info.ndof, 2), dtype=torch.float64, device="cuda")
        n, _ = ibem.ibem_solver_residuals(h, b, 2, r, rtol=1e-10, maxit=400, stride=1, max_vecs=60)
        l0 = ibem.ibem_cnn_operator_gradients(h, c, r[:min(n, 64)].contiguous(), min(n, 64), ibem.IBEM_BF16,
                                              ibem.IBEM_FP32)[0]
        l1 = ibem.ibem_cnn_train_operator(h, c, r, n, batch=16, epochs=8, lr=1e-3, seed=len(train))
        train.append({"k": float(k), "vectors": n, "objective_before": l0, "objective_after": l1})
        ibem.ibem_destroy(h)
    train_s = time.perf_counter() - t0
    k = float(rng.uniform(8.0, 16.0))
    h = make(args.learn_m, k)
    info = ibem.ibem_get_info(h)
    b = plane_rhs(h, k, args.learn_nrhs)
    w = torch.empty_like(b)
    res = {}
    for name, pc in (("block_jacobi", ibem.IBEM_PRECOND_BLOCK_JACOBI), ("learned", ibem.IBEM_PRECOND_LEARNED)):
        ibem.ibem_set_learned_preconditioner(h, c if pc == ibem.IBEM_PRECOND_LEARNED else None)
        s, si = ibem.ibem_solve(h, b, w, args.learn_nrhs, rtol=1e-8, maxit=3000, precond=pc, check=False)
        res[name] = {"status": ibem.ibem_status_string(s), "iterations": si.iterations,
                     "rel_residual_fp64": si.rel_residual, "seconds": si.seconds}
    ibem.ibem_set_learned_preconditioner(h, None)
    ibem.ibem_destroy(h)
    fwd = cnn_forward_timing(ibem, stream, c)
    ibem.ibem_cnn_destroy(c)
    it_b, it_l = res["block_jacobi"]["iterations"], res["learned"]["iterations"]
    return {"workload": "helmholtz-sphere-p2-q6-k[8,16]: train level %d, solve level %d, %d plane waves"
                        % (args.learn_train_m, args.learn_m, args.learn_nrhs),
            "k_solve": k, "ndof": info.ndof, "train": train, "train_s": train_s, "solve": res,
            "iterations_learned_over_block_jacobi": it_l / max(1, it_b),
            "seconds_learned_over_block_jacobi": res["learned"]["seconds"] / max(1e-9, res["block_jacobi"]["seconds"]),
            "cnn_forward": fwd}


# ---------------------------------------------------------------- our arm
def ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_1708_09162_gb300 import build
    build.build()
    from paper_1708_09162_gb300 import ibem

    torch.cuda.set_device(local_rank)
    dist = world > 1
    if dist:
        import torch.distributed as td

    def barrier():
        if dist:
            td.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.Stream()
    if args.helmholtz_many_only:
        out = helmholtz_many_rhs(ibem, stream, world, barrier, args)
        if rank == 0:
            print(json.dumps({"helmholtz_64rhs": out}), flush=True)
        return
    if args.batch_only:
        out = batched_instances(ibem, stream, args)
        if rank == 0:
            print(json.dumps({"batched_instances": out}), flush=True)
        return
    if args.cnn_forward_only:
        c = ibem.ibem_cnn_create(32, seed=SEED, stream=stream)
        out = cnn_forward_timing(ibem, stream, c)
        ibem.ibem_cnn_destroy(c)
        if rank == 0:
            print(json.dumps({"cnn_forward": out}), flush=True)
        return
    if args.learned_only:
        out = learned_preconditioner(ibem, stream, args)
        if rank == 0:
            print(json.dumps({"learned_preconditioner": out}), flush=True)
        return
    prm = ibem.make_params(WORKLOAD["p"], WORKLOAD["m"], q_cheb=WORKLOAD["q_cheb"], eta=WORKLOAD["eta"])
    t0 = time.perf_counter()
    h = ibem.ibem_create(ibem.sphere_patches(), prm, stream)
    t_create = time.perf_counter() - t0
    t0 = time.perf_counter()
    ibem.ibem_assemble(h)
    t_assemble = time.perf_counter() - t0
    info = ibem.ibem_get_info(h)
    N, R = info.ndof, WORKLOAD["nrhs"]
    rng = np.random.default_rng(SEED + rank)
    x = torch.from_numpy(rng.normal(size=(R, N))).cuda()
    y = torch.empty_like(x)
    y32 = torch.empty_like(x)

    def run(steps, precision):
        with torch.cuda.stream(stream):
            for _ in range(steps):
                ibem.ibem_matvec(h, x, y if precision == 0 else y32, R, precision)

    # ---- FP64 operator: the headline ----
    run(args.warmup, 0)
    ibem.ibem_profile_read(h)
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ibem.ibem_profile_enable(h, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    run(args.steps, 0)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = ibem.ibem_profile_read(h)
    ibem.ibem_profile_enable(h, False)
    clk = clocks.stop()
    ms = max_over_ranks(ms)
    value = job_throughput(world, N * R, ms * 1e-3)

    # ---- roofline of the dominant kernel ----
    # coupling_df_kernel streams the double-float coupling matrices (8 bytes per
    # entry) once and spends 12 FP32-pipe operations per entry (exact product,
    # two cross terms, TwoSum); its bound is whichever fraction is larger.
    phase_ms = {k: v / args.steps for k, v in prof["ms"].items()}
    q2 = WORKLOAD["q_cheb"] ** 2
    kpt = (q2 + 3) // 4
    coup_ms = phase_ms["coupling"]
    entries = float(q2 * q2 * info.n_far * R)          # matrix entries applied (both halves)
    # bytes: the stored upper half of K (symmetric storage), the source moments
    # streamed with every block, column shares written and gathered, y^ written
    n_up = info.bytes_far // (kpt * 4 * q2 * 8)
    kbytes = info.bytes_far + n_up * ((q2 + 1) // 2 * 2) * 8 * R + n_up * q2 * 8 * R + \
        info.n_clusters * q2 * R * 8
    hbm_gbs, sm_max, peak_src = _peaks()
    fp32_peak_tops = 152 * 128 * sm_max * 1e6 / 1e12            # FP32 lanes x clock
    alu_frac = (12.0 * entries / (coup_ms * 1e-3) / 1e12) / fp32_peak_tops
    hbm_frac = (kbytes / (coup_ms * 1e-3) / 1e9) / hbm_gbs
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": 12.0 * entries / (coup_ms * 1e-3) / 1e12, "peak": fp32_peak_tops,
                "unit": "Tops/s", "frac": alu_frac,
                "peak_source": "FP32 pipe: 152 SMs x 128 lanes x %.0f MHz (%s clock)" % (sm_max, peak_src)}
    else:
        roof = {"bound": "hbm", "achieved": kbytes / (coup_ms * 1e-3) / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                "frac": hbm_frac, "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s; of measured)" % peak_src}
    roof.update({"kernel": "coupling_df_kernel", "ms_per_launch": coup_ms, "traffic": _profile_traffic(),
                 "algorithmic_bytes": kbytes, "matrix_entries": entries, "flops_equiv_fp64": 2.0 * entries,
                 "hbm_frac_of_measured": hbm_frac, "fp32_alu_frac": alu_frac})

    # ---- native FP64 coupling (FP64 FMA pipe), for comparison ----
    native = None
    if not args.no_native:
        hn = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(
            WORKLOAD["p"], WORKLOAD["m"], q_cheb=WORKLOAD["q_cheb"], eta=WORKLOAD["eta"],
            fp64_coupling=ibem.IBEM_COUPLING_NATIVE), stream)
        ibem.ibem_assemble(hn)
        yn = torch.empty_like(x)
        nsteps = max(3, args.steps // 4)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                ibem.ibem_matvec(hn, x, yn, R, 0)
        barrier()
        ibem.ibem_profile_enable(hn, True)
        ev0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(nsteps):
                ibem.ibem_matvec(hn, x, yn, R, 0)
        ev1.record(stream)
        barrier()
        pn = ibem.ibem_profile_read(hn)
        msn = ev0.elapsed_time(ev1) / nsteps
        native = {"value": world * N * R / (msn * 1e-3), "ms_per_step": msn,
                  "coupling_ms": pn["ms"]["coupling"] / nsteps,
                  "rel_diff_vs_double_float": float((yn - y).abs().max() / y.abs().max())}
        ibem.ibem_destroy(hn)

    # ---- FP32 operator ----
    run(args.warmup, 1)
    barrier()
    ev0.record(stream)
    run(args.steps, 1)
    ev1.record(stream)
    barrier()
    ms32 = ev0.elapsed_time(ev1) / args.steps
    err32 = float((y32 - y).abs().max() / y.abs().max())

    # ---- end to end through the host-buffer entry point ----
    xh = torch.empty((R, N), dtype=torch.float64, pin_memory=True)
    xh.copy_(x.cpu())
    yh = torch.empty((R, N), dtype=torch.float64, pin_memory=True)
    e2e_steps = max(3, args.steps // 10)
    for _ in range(3):
        ibem.ibem_matvec_host(h, xh, yh, R)
    barrier()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        ibem.ibem_matvec_host(h, xh, yh, R)
    e2e_s = (time.perf_counter() - t) / e2e_steps
    e2e_s = max_over_ranks(e2e_s)

    # ---- solves to 1e-8 ----
    solve = None
    if not args.no_solve:
        x0 = np.array([0.9, 0.9, 0.9])
        qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
        ibem.ibem_quad_points(h, qp)
        torch.cuda.synchronize()
        gq = torch.from_numpy(1.0 / (4 * np.pi * np.linalg.norm(qp.cpu().numpy() - x0, axis=1))).cuda()
        b = torch.empty(N, dtype=torch.float64, device="cuda")
        ibem.ibem_rhs(h, gq, 1, b)
        w = torch.empty_like(b)
        solve = {"rtol": 1e-8, "rhs": "point source 1/(4 pi |x - x0|), x0 = (0.9, 0.9, 0.9)"}
        for name, pc in (("jacobi", ibem.IBEM_PRECOND_JACOBI), ("block_jacobi", ibem.IBEM_PRECOND_BLOCK_JACOBI)):
            s64 = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=5000, precond=pc, precision=0)
            s32 = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=5000, precond=pc, precision=1)
            solve[name] = {"fp64": {"seconds": s64.seconds, "iterations": s64.iterations,
                                    "rel_residual": s64.rel_residual},
                           "mixed": {"seconds": s32.seconds, "iterations": s32.iterations,
                                     "fp64_updates": s32.outer, "rel_residual": s32.rel_residual},
                           "speedup_mixed_vs_fp64": s64.seconds / s32.seconds}

    # ---- Helmholtz, 64 plane waves: tensor-core coupling ----
    helm_many = None if args.no_helmholtz_many else helmholtz_many_rhs(ibem, stream, world, barrier, args)

    # ---- many uneven instances in one application ----
    batched = None if args.no_batch else batched_instances(ibem, stream, args)

    # ---- learned preconditioner vs block-Jacobi ----
    learned = None if args.no_learned else learned_preconditioner(ibem, stream, args)

    # ---- oracle on the host cores (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        o = run_oracle(3)
        cpu = {"value": o["rows"] / o["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d rows of the oracle's FMM-mode operator on the same workload (near blocks, "
                         "far couplings and the moment pass included; tree setup %.1f s excluded)"
                         % (o["rows"], o["setup_s"])}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, ndof=N, ndof_super=info.ndof_super, n_near=info.n_near, n_far=info.n_far,
                           parallelism="replicas" if world > 1 else "single",
                           l2="inputs larger than L2: %.1f GB of stored operator streamed per step"
                              % ((info.bytes_near + info.bytes_far) / 1e9)),
            "phase_ms": phase_ms,
            "fp32": {"value": world * N * R / (ms32 * 1e-3), "ms_per_step": ms32, "rel_err_vs_fp64": err32},
            "fp64_native_coupling": native,
            "assemble_s": t_assemble, "create_s": t_create,
            "solve": solve,
            "roofline": roof,
            "cpu_baseline": cpu,
            "helmholtz_64rhs": helm_many,
            "learned_preconditioner": learned,
            "batched_instances": batched,
            "e2e": {"value": world * N * R / e2e_s, "unit": UNIT, "h2d_bytes_per_step": N * R * 8,
                    "d2h_bytes_per_step": N * R * 8},
            "gpu_launches": prof["launches"],
            "clocks": clk}
    ibem.ibem_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.m is not None:
        WORKLOAD["m"] = args.m
        WORKLOAD["workload"] = "laplace-sphere-p%d-m%d-q%d-eta%g" % (WORKLOAD["p"], args.m, WORKLOAD["q_cheb"],
                                                                    WORKLOAD["eta"])
    if args.oracle_worker:
        oracle_worker(args.oracle_worker)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl")
    ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
