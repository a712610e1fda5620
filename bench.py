#!/usr/bin/env python3
"""Benchmark of the FMM-compressed single-layer operator on one GB300.

Headline workload (Helmholtz sound-soft scattering): the unit sphere as 6
cube-sphere patches, degree-2 B-splines on level 6 (26,136 complex dofs,
221,184 superspace dofs), Chebyshev 8 x 8 points per cluster, admissibility
eta = 1.6, wavenumber kappa = 4, 64 right-hand sides.

A step is one application of y = T A T^T x to all 64 right-hand sides (lift,
upward pass, coupling, downward pass, near field, restriction) with the
FP64-accurate operator: FP64 near blocks and the coupling generated per far
block in double-float arithmetic and contracted on the tensor cores as exact
products of BF16 digit slices, recombined in double-float (about 45
significant bits; --coupling generate contracts in double-float on the FP32
pipe instead).  `value` is dofs x right-hand sides per second over all
ranks (each rank runs an independent replica; no data-path collective).
Beside it: the FP32 operator with the coupling on the tensor cores, both
operators' errors against the oracle on sampled rows at full size, the
lock-step GMRES solves of the 64 plane waves to true relative residual 1e-8
(mixed precision against plain FP64), the end-to-end time through
ibem_matvec_host with host buffers, the Laplace degree-3 workload on level 5,
the batched instances, the learned preconditioner, the roofline of the
dominant kernel and the oracle on all host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "helmholtz-sphere-p2-m6-q8-k4-R64", "kernel": "helmholtz", "kappa": 4.0, "p": 2, "m": 6,
            "q_cheb": 8, "eta": 1.6, "nrhs": 64, "geometry": "unit sphere, 6 cube-sphere patches",
            "rhs": "64 sound-soft plane waves, directions seeded uniform on S^2",
            "coupling": "generated per far block in double-float, contracted in BF16 digit slices on the "
                        "tensor cores (exact FP32 accumulation) or in double-float (--coupling generate)"}
LAPLACE = {"workload": "laplace-sphere-p3-m5-q6-eta1.6", "p": 3, "m": 5, "q_cheb": 6, "eta": 1.6, "nrhs": 1}
METRIC = "FMM single-layer matvec DOF·RHS/s and GMRES solve time to 1e-8, vs plain FP64 GPU"
UNIT = "DOF*RHS/s"
SEED = 170809162
ORACLE_ROWS = 32          # sampled rows of the oracle's FMM-mode operator (one right-hand side)
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "helm_coupling_sliced_kernel_helmholtz_sphere_p2_k4.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=None, help="refinement level override (profiling cases)")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-fp64-solve", action="store_true", help="skip the plain FP64 solve")
    ap.add_argument("--no-store", action="store_true", help="skip the stored-BF16 coupling section")
    ap.add_argument("--coupling", choices=("generate", "sliced"), default="sliced",
                    help="FP64-accurate coupling of the headline operator: double-float on the FP32 pipe, or "
                         "BF16 digit slices on the tensor cores")
    ap.add_argument("--fp32-store", action="store_true", help="with --fp32-only: time the stored-BF16 coupling")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-laplace", action="store_true", help="skip the Laplace level-5 section")
    ap.add_argument("--no-potential", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner section")
    ap.add_argument("--learned-only", action="store_true", help="run only the learned-preconditioner section")
    ap.add_argument("--config4", action="store_true",
                    help="run only the 256-instance batched workload (several minutes of setup)")
    ap.add_argument("--fmm-error-study", action="store_true",
                    help="run only the FMM-against-dense error study of the Laplace level-5 workload")
    ap.add_argument("--learned-config5", action="store_true",
                    help="run only the learned preconditioner at level 7 with 16 plane waves (several minutes)")
    ap.add_argument("--cnn-forward-only", action="store_true", help="time only the network's forward pass")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances section")
    ap.add_argument("--batch-only", action="store_true", help="run only the batched-instances section")
    ap.add_argument("--operator-only", action="store_true",
                    help="headline operator only (profiling): no solves, side sections or oracle")
    ap.add_argument("--fp32-only", action="store_true", help="time only the tensor-core FP32 operator (profiling)")
    ap.add_argument("--laplace-only", action="store_true", help="run only the Laplace level-5 section (profiling)")
    ap.add_argument("--learn-train-m", type=int, default=5, help="level of the training solves")
    ap.add_argument("--learn-m", type=int, default=6, help="level of the compared solves")
    ap.add_argument("--learn-nrhs", type=int, default=2, help="plane waves of the compared solves")
    ap.add_argument("--oracle-child", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def sampled_input(n):
    """The seeded input of the accuracy checks and the oracle sample: rows and one
    complex right-hand side (normal real and imaginary parts)."""
    import numpy as np
    rng = np.random.default_rng(SEED + 11)
    rows = np.sort(rng.choice(n, size=ORACLE_ROWS, replace=False))
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    return rows, x


# ---------------------------------------------------------------- oracle (CPU)
def _oracle_op():
    from oracle import fmm, galerkin, geometry
    disc = galerkin.Discretisation(geometry.unit_sphere(), WORKLOAD["p"], WORKLOAD["m"],
                                   galerkin.HelmholtzKernel(WORKLOAD["kappa"]))
    return fmm.FMMOperator(disc, WORKLOAD["q_cheb"], WORKLOAD["eta"])


_OP = None


def _rows_task(chunk):
    import numpy as np
    rows, x = chunk
    t = time.perf_counter()
    y = _OP.rows([int(r) for r in rows], x)[:, 0]
    return np.stack([y.real, y.imag], -1).tolist(), time.perf_counter() - t


def oracle_child(path):
    """Runs in a fresh CPU-only process (no CUDA): builds the oracle's FMM-mode
    operator of the headline workload once, then computes ORACLE_ROWS sampled
    rows of A x for one seeded right-hand side in a pool of one worker per host
    core (forked after the build, so the workers share the operator); the
    timed region is the pool's row phase.  Writes one JSON file."""
    import multiprocessing as mp
    import numpy as np
    global _OP
    t0 = time.perf_counter()
    _OP = _oracle_op()
    setup = time.perf_counter() - t0
    n = _OP.mesh.n_dofs
    rows, x = sampled_input(n)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    chunks = [(rows[i::cores], x) for i in range(min(cores, len(rows)))]
    ctx = mp.get_context("fork")
    t = time.perf_counter()
    with ctx.Pool(len(chunks)) as pool:
        res = pool.map(_rows_task, chunks, chunksize=1)
    wall = time.perf_counter() - t
    y = np.zeros((len(rows), 2))
    for i, (vals, _) in enumerate(res):
        y[i::len(chunks)] = np.array(vals)
    json.dump({"rows": rows.tolist(), "y": y.tolist(), "seconds": wall, "setup_s": setup,
               "workers": len(chunks), "cores": cores, "cpu": cpu_model(),
               "busy_s": sum(r[1] for r in res)}, open(path, "w"))


def start_oracle_child():
    fd, path = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-child", path], env=env, cwd=ROOT,
                            stdout=subprocess.DEVNULL, stderr=subprocess.PIPE, text=True)
    return proc, path


def finish_oracle_child(proc, path):
    _, err = proc.communicate()
    if proc.returncode != 0:
        raise RuntimeError("oracle child failed: " + (err or "")[-2000:])
    with open(path) as f:
        d = json.load(f)
    os.unlink(path)
    return d


def reference_arm(args, rank):
    """The oracle, as it stands, on the host cores: a pool of one worker per core
    (forked after the operator's tree is built once, outside the steps); each
    step computes one sampled row of the FMM-mode operator of the headline
    workload per worker, applied to one right-hand side."""
    if rank != 0:
        return
    import multiprocessing as mp
    import numpy as np
    global _OP
    t0 = time.perf_counter()
    _OP = _oracle_op()
    setup = time.perf_counter() - t0
    n = _OP.mesh.n_dofs
    rng = np.random.default_rng(SEED)
    _, x = sampled_input(n)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    with mp.get_context("fork").Pool(cores) as pool:
        def step():
            pool.map(_rows_task, [(rng.choice(n, 1), x) for _ in range(cores)], chunksize=1)

        for _ in range(args.warmup):
            step()
        t = time.perf_counter()
        for _ in range(args.steps):
            step()
        dt = time.perf_counter() - t
    value = args.steps * cores / dt
    cfg = dict(WORKLOAD, ndof=n, ndof_super=_OP.mesh.n_elements * (WORKLOAD["p"] + 1) ** 2, n_near=len(_OP.near),
               n_far=len(_OP.far), parallelism="single")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": "per step one sampled row of the oracle's FMM-mode operator per core, one "
                                       "right-hand side, near blocks and the moments the rows use included "
                                       "(tree setup %.0f s excluded); one BLAS thread per worker" % setup},
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
            "launches_per_apply": info["launches_per_apply"], "coupling_threads": info["coupling_threads"],
            "coupling_rhs_tile": info["coupling_rhs_tile"]}


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


def bessel_zeros(lmax, lo, hi):
    """Zeros of the spherical Bessel functions j_l, l <= lmax, in [lo, hi]
    (sign changes on a fine grid, refined by Brent's method)."""
    import numpy as np
    from scipy import optimize, special
    zs = []
    g = np.linspace(lo, hi, 4001)
    for l in range(lmax + 1):
        v = special.spherical_jn(l, g)
        for i in np.nonzero(np.sign(v[:-1]) * np.sign(v[1:]) < 0)[0]:
            zs.append(optimize.brentq(lambda t: special.spherical_jn(l, t), g[i], g[i + 1]))
    return np.array(sorted(zs))


def draw_wavenumbers(rng, n, lo=8.0, hi=16.0, gap=0.02, lmax=20):
    """n wavenumbers uniform in [lo, hi], rejecting draws within `gap` of a zero
    of j_l (l <= lmax): there the single-layer operator of the unit sphere has a
    vanishing eigenvalue.  Returns the kept and the rejected draws."""
    import numpy as np
    zeros = bessel_zeros(lmax, lo - 1.0, hi + 1.0)
    kept, rejected = [], []
    while len(kept) < n:
        k = float(rng.uniform(lo, hi))
        (rejected if np.min(np.abs(zeros - k)) < gap else kept).append(k)
    return kept, rejected


def learned_config5(ibem, stream, args):
    """Learned preconditioner at the 101,400-dof workload: Helmholtz sound-soft
    scattering on the unit sphere, p = 2, level 7, q = 8, kappa drawn uniformly
    from [8, 16] (resonance filter: no draw within 0.02 of a zero of j_l,
    l <= 20), 16 seeded plane waves.  Two networks (4 layers, 32 channels, BF16)
    are trained on the plain solver's residuals at levels 5 and 6 (q = 6, three
    wavenumbers each, two plane waves, residual-norm objective): one on the fine
    coefficient images, one on the coarse grid with f = 2^(m - 4) (the level-4
    grid at every level).  Lock-step flexible GMRES(100) with each is compared
    with block-Jacobi GMRES(100), all with the FP32 operator (tensor-core
    coupling) inside iterative refinement and measured by the FP64 true residual
    1e-8 of every right-hand side."""
    import numpy as np
    import torch
    rng = np.random.default_rng(SEED + 13)
    k_solve, rejected = draw_wavenumbers(rng, 1)
    k_solve = k_solve[0]

    def make(m, q, k, coupling=0):
        h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(2, m, q_cheb=q, eta=1.6,
                                                                     kernel=ibem.IBEM_HELMHOLTZ, kappa=k,
                                                                     fp64_coupling=coupling), stream)
        ibem.ibem_assemble(h)
        return h

    nets = {"fine": ibem.ibem_cnn_create(32, seed=SEED, stream=stream),
            "coarse": ibem.ibem_cnn_create(32, seed=SEED, stream=stream)}
    t0 = time.perf_counter()
    train = []
    for m in (5, 6):
        ks, rej = draw_wavenumbers(rng, 3)
        rejected += rej
        for k in ks:
            h = make(m, 6, k)
            info = ibem.ibem_get_info(h)
            b = plane_wave_rhs(ibem, h, k, 2, int(rng.integers(1 << 30)))
            r = torch.zeros((2 * 60, info.ndof, 2), dtype=torch.float64, device="cuda")
            _, n, _ = ibem.ibem_solver_residuals(h, b, 2, r, rtol=1e-10, maxit=600, stride=1, max_vecs=60,
                                                 check=False)
            rec = {"level": m, "k": k, "vectors": n}
            for name, c in nets.items():
                ibem.ibem_cnn_set_coarsening(c, 2 ** (m - 4) if name == "coarse" else 1)
                rec["objective_after_" + name] = ibem.ibem_cnn_train_operator(h, c, r, n, batch=16, epochs=6,
                                                                              lr=1e-3, seed=len(train))
            train.append(rec)
            ibem.ibem_destroy(h)
    train_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    h = make(7, 8, k_solve, ibem.IBEM_COUPLING_GENERATE)
    setup_s = time.perf_counter() - t0
    info = ibem.ibem_get_info(h)
    R = 16
    b = plane_wave_rhs(ibem, h, k_solve, R, SEED + 14)
    ibem.ibem_cnn_set_coarsening(nets["coarse"], 2 ** (7 - 4))
    res = {}
    for name, pc, c in (("block_jacobi", ibem.IBEM_PRECOND_BLOCK_JACOBI, None),
                        ("learned_fine", ibem.IBEM_PRECOND_LEARNED, nets["fine"]),
                        ("learned_coarse", ibem.IBEM_PRECOND_LEARNED, nets["coarse"])):
        ibem.ibem_set_learned_preconditioner(h, c)
        w = torch.empty_like(b)
        s, si = ibem.ibem_solve(h, b, w, R, rtol=1e-8, maxit=4000, precond=pc, precision=ibem.IBEM_FP32,
                                check=False)
        res[name] = {"status": ibem.ibem_status_string(s), "steps": si.steps, "iterations": si.iterations,
                     "outer": si.outer, "rel_residual_fp64": si.rel_residual, "seconds": si.seconds}
    ibem.ibem_set_learned_preconditioner(h, None)
    ibem.ibem_destroy(h)
    for c in nets.values():
        ibem.ibem_cnn_destroy(c)
    bjs = max(1, res["block_jacobi"]["steps"])
    return {"workload": "helmholtz-sphere-p2-m7-q8-R16, kappa from [8, 16]", "k_solve": k_solve,
            "k_rejected_by_filter": rejected, "ndof": info.ndof, "n_far": info.n_far, "setup_s": setup_s,
            "train": train, "train_s": train_s, "solve": res,
            "steps_over_block_jacobi": {k: v["steps"] / bjs for k, v in res.items()}}


def config4_section(ibem, stream, args):
    """The batched-instances workload at its full size: 256 seeded instances, each
    the 6-patch sphere with radius uniform in [0.5, 2], level 3-6 and degree 1-3
    uniform, Laplace (first half, q = 6) or Helmholtz with kappa uniform in
    [1, 8] (second half, q = 8), 1-16 right-hand sides; FP32-only handles (the
    FP64 near blocks are released after assembly).  The batched, graph-captured
    application (one launch per stage, persistent coupling kernel with autotuned
    tile and CTA size) is timed against the same instances applied one after
    another through ibem_matvec, and each instance's batched result is compared
    with its own application."""
    import numpy as np
    import torch
    rng = np.random.default_rng(SEED + 40)
    n = 256
    specs = []
    for i in range(n):
        helm = i >= n // 2
        specs.append({"kernel": int(helm), "p": int(rng.integers(1, 4)), "m": int(rng.integers(3, 7)),
                      "R": int(rng.integers(1, 17)), "radius": float(rng.uniform(0.5, 2.0)),
                      "kappa": float(rng.uniform(1.0, 8.0)) if helm else 0.0, "q": 8 if helm else 6})
    handles, setup = [], {}
    t0 = time.perf_counter()
    for sp in specs:
        t = time.perf_counter()
        h = ibem.ibem_create(ibem.sphere_patches(sp["radius"]), ibem.make_params(
            sp["p"], sp["m"], q_cheb=sp["q"], kernel=sp["kernel"], kappa=sp["kappa"],
            fp64_coupling=ibem.IBEM_COUPLING_FP32_ONLY), stream)
        ibem.ibem_assemble(h)
        handles.append(h)
        setup[sp["m"]] = setup.get(sp["m"], 0.0) + time.perf_counter() - t
    setup_s = time.perf_counter() - t0
    nrhs = [sp["R"] for sp in specs]
    dofs = sum(ibem.ibem_get_info(h).ndof * R for h, R in zip(handles, nrhs))
    t = time.perf_counter()
    b = ibem.ibem_batch_create(handles, nrhs, stream)
    create_s = time.perf_counter() - t
    off = ibem.ibem_batch_offsets(b, n)
    x = torch.from_numpy(rng.normal(size=off[-1])).cuda()
    y, ys = torch.zeros_like(x), torch.zeros_like(x)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        with torch.cuda.stream(stream):
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

    batched_ms = timed(lambda: ibem.ibem_batch_matvec(b, x, y), 5)
    single_ms = timed(one_by_one, 3)
    worst = 0.0
    for i in range(n):
        a, c = y[off[i]:off[i + 1]], ys[off[i]:off[i + 1]]
        worst = max(worst, float((a - c).abs().max() / c.abs().max()))
    info = ibem.ibem_batch_info(b)
    mem = torch.cuda.mem_get_info()
    ibem.ibem_batch_destroy(b)
    for h in handles:
        ibem.ibem_destroy(h)
    return {"instances": n, "dof_rhs_per_apply": dofs, "setup_s": setup_s,
            "setup_s_by_level": {str(k): v for k, v in sorted(setup.items())}, "batch_create_s": create_s,
            "batched_ms": batched_ms, "one_by_one_ms": single_ms, "speedup": single_ms / batched_ms,
            "value": dofs / (batched_ms * 1e-3), "unit": UNIT, "max_rel_diff_batched_vs_own": worst,
            "launches_per_apply": info["launches_per_apply"], "coupling_threads": info["coupling_threads"],
            "coupling_rhs_tile": info["coupling_rhs_tile"],
            "device_memory_used_gb": (mem[1] - mem[0]) / 1e9,
            "levels": {str(m): sum(1 for sp in specs if sp["m"] == m) for m in range(3, 7)}}


def fmm_error_study(ibem, stream, args):
    """FMM error of the Laplace degree-3 level-5 workload (q = 6, eta = 1.6)
    against the dense Galerkin matrix of the same quadrature (every element
    pair as near field), for both readings of the admissibility condition
    (Def. 4.1): eta max(diam) < dist (the default) and max(diam) < eta dist.
    Operator applied to one seeded vector and to the point-source right-hand
    side; max-norm relative errors over all dofs."""
    import numpy as np
    import torch
    W = LAPLACE
    x = torch.from_numpy(np.random.default_rng(SEED + 21).normal(size=(1, 7350))).cuda()
    out = {"workload": W["workload"]}
    t0 = time.perf_counter()
    hd = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(W["p"], W["m"], q_cheb=0), stream)
    ibem.ibem_assemble(hd)
    out["dense_setup_s"] = time.perf_counter() - t0
    info = ibem.ibem_get_info(hd)
    out["dense_near_pairs"] = info.n_near
    yd = torch.empty_like(x)
    ibem.ibem_matvec(hd, x, yd, 1, 0)
    torch.cuda.synchronize()
    ibem.ibem_destroy(hd)
    for name, adm in (("eta_max_diam_lt_dist", ibem.IBEM_ADMISSIBLE_ETA_DIAM),
                      ("max_diam_lt_eta_dist", ibem.IBEM_ADMISSIBLE_ETA_DIST)):
        for q in (4, 6, 8):
            h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(W["p"], W["m"], q_cheb=q, eta=W["eta"],
                                                                         admissibility=adm), stream)
            ibem.ibem_assemble(h)
            inf = ibem.ibem_get_info(h)
            y = torch.empty_like(x)
            ibem.ibem_matvec(h, x, y, 1, 0)
            torch.cuda.synchronize()
            out["%s_q%d" % (name, q)] = {"n_near": inf.n_near, "n_far": inf.n_far,
                                         "rel_err_vs_dense": float((y - yd).abs().max() / yd.abs().max())}
            ibem.ibem_destroy(h)
    return out


def _peak_tensor():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f).get("bf16_tflops", 1912.6), "measured"
    except OSError:
        return 1900.0, "fallback"


def gen_ops_per_launch(n_far, q, R):
    """FP32-pipe operations of the double-float coupling, counted from its
    formulas: 247 per generated complex kernel value (differences, r^2, r, 1/r,
    the phase and its reduction, the Taylor terms, the table product) and 48 per
    complex multiply-add and right-hand side (four exact products with their
    error terms and TwoSum accumulations of 12 operations each)."""
    q4 = float(q) ** 4
    return n_far * q4 * 247.0, n_far * q4 * 48.0 * R


def sliced_ops_per_launch(n_far, R):
    """FP32-pipe operations of the digit-sliced coupling (q = 8), counted from its
    formulas per far block and chunk of 32 right-hand sides: 247 per generated
    complex kernel value (as the double-float coupling), 58 per sliced real
    value (scaling, and per each of 6 digits: rint, the exact remainder with a
    Fast2Sum, the rescaling and the BF16 packing) and 48 per recombined
    accumulator entry (the FP32 and double-float Horner steps over 6 levels, the
    power-of-two scale and the double-float row sum); and the tensor work, 21
    slice pairs of 2 x 128 x 64 x 64 flops."""
    nch = (R + 31) // 32
    per = 4096 * 247.0 + 8192 * 58.0 + 8192 * 48.0
    return n_far * nch * per, n_far * nch * 21 * 2.0 * 128 * 64 * 64


def plane_wave_rhs(ibem, h, kappa, R, seed):
    import numpy as np
    import torch
    info = ibem.ibem_get_info(h)
    d = np.random.default_rng(seed).normal(size=(R, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    torch.cuda.synchronize()
    g = -np.exp(1j * kappa * (d @ qp.cpu().numpy().T))          # sound-soft data, [R, nq]
    gq = torch.from_numpy(np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))).cuda()
    b = torch.empty((R, info.ndof, 2), dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, gq, R, b)
    return b


def laplace_section(ibem, stream, world, barrier, steps, warmup):
    """The Laplace workload of the previous headline: p = 3, m = 5, q = 6, one
    right-hand side, FP64 operator with the stored symmetric double-float
    coupling (HBM-bound), FP32 operator, block-Jacobi CG FP64 and mixed."""
    import numpy as np
    import torch
    W = LAPLACE
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(W["p"], W["m"], q_cheb=W["q_cheb"], eta=W["eta"]),
                         stream)
    t0 = time.perf_counter()
    ibem.ibem_assemble(h)
    asm = time.perf_counter() - t0
    info = ibem.ibem_get_info(h)
    N = info.ndof
    x = torch.from_numpy(np.random.default_rng(SEED).normal(size=(1, N))).cuda()
    y, y32 = torch.empty_like(x), torch.empty_like(x)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(prec, out, n):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                ibem.ibem_matvec(h, x, out, 1, prec)
        barrier()
        ibem.ibem_profile_enable(h, True)
        ev0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(n):
                ibem.ibem_matvec(h, x, out, 1, prec)
        ev1.record(stream)
        barrier()
        prof = ibem.ibem_profile_read(h)
        ibem.ibem_profile_enable(h, False)
        return ev0.elapsed_time(ev1) / n, {k: v / n for k, v in prof["ms"].items()}

    ms, ph = timed(0, y, steps)
    ms32, _ = timed(1, y32, steps)
    # roofline of coupling_df_kernel: the stored upper half of K (8 bytes per
    # double-float entry), the moments streamed with every block, column shares
    # written and gathered, y^ written
    q2 = W["q_cheb"] ** 2
    kpt = (q2 + 3) // 4
    n_up = info.bytes_far // (kpt * 4 * q2 * 8)
    kbytes = info.bytes_far + n_up * ((q2 + 1) // 2 * 2) * 8 + n_up * q2 * 8 + info.n_clusters * q2 * 8
    hbm, _, src = _peaks()
    coup = ph["coupling"]
    x0 = np.array([0.9, 0.9, 0.9])
    qp = torch.empty((info.n_quad_points, 3), dtype=torch.float64, device="cuda")
    ibem.ibem_quad_points(h, qp)
    torch.cuda.synchronize()
    gq = torch.from_numpy(1.0 / (4 * np.pi * np.linalg.norm(qp.cpu().numpy() - x0, axis=1))).cuda()
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    ibem.ibem_rhs(h, gq, 1, b)
    w = torch.empty_like(b)
    s64 = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=5000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI, precision=0)
    s32 = ibem.ibem_solve(h, b, w, 1, rtol=1e-8, maxit=5000, precond=ibem.IBEM_PRECOND_BLOCK_JACOBI, precision=1)
    ibem.ibem_destroy(h)
    return {"workload": W["workload"], "ndof": N, "ndof_super": info.ndof_super, "n_near": info.n_near,
            "n_far": info.n_far, "assemble_s": asm,
            "fp64": {"value": world * N / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "phase_ms": ph,
                     "dtype": "f64 (stored double-float coupling, about 48 bits)"},
            "fp32": {"value": world * N / (ms32 * 1e-3), "ms_per_step": ms32,
                     "rel_err_vs_fp64": float((y32 - y).abs().max() / y.abs().max())},
            "roofline_coupling": {"kernel": "coupling_df_kernel", "bound": "hbm", "algorithmic_bytes": kbytes,
                                  "achieved": kbytes / (coup * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                                  "frac": kbytes / (coup * 1e-3) / 1e9 / hbm,
                                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % src},
            "block_jacobi_cg": {"rtol": 1e-8, "rhs": "point source 1/(4 pi |x - x0|), x0 = (0.9, 0.9, 0.9)",
                                "fp64": {"seconds": s64.seconds, "iterations": s64.iterations,
                                         "rel_residual": s64.rel_residual},
                                "mixed": {"seconds": s32.seconds, "iterations": s32.iterations,
                                          "fp64_updates": s32.outer, "rel_residual": s32.rel_residual},
                                "speedup_mixed_vs_fp64": s64.seconds / s32.seconds}}


def potentials_section(ibem, stream, h, b):
    """Potentials of the 64 densities (the right-hand sides stand in for them) at
    200 seeded points on the sphere of radius 3: direct Gauss sums (FP64) and with
    the far field interpolated."""
    import numpy as np
    import torch
    info = ibem.ibem_get_info(h)
    R = b.shape[0]
    npt = 200
    dp = np.random.default_rng(SEED + 4).normal(size=(npt, 3))
    pts = torch.from_numpy(3.0 * dp / np.linalg.norm(dp, axis=1)[:, None]).cuda()
    u = torch.empty((R, npt, 2), dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ibem.ibem_potential(h, b, R, pts, u)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(2):
            ibem.ibem_potential(h, b, R, pts, u)
    e1.record(stream)
    torch.cuda.synchronize()
    pot_ms = e0.elapsed_time(e1) / 2
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
    nsrc = info.n_elements * 64
    return {"points": npt, "densities": R, "sources": nsrc, "direct_ms": pot_ms,
            "pair_density_evals_per_s": npt * nsrc * R / (pot_ms * 1e-3),
            "interpolated": {"ms": fmm_ms, "far_terms": nf, "near_terms": nn, "speedup": pot_ms / fmm_ms,
                             "rel_err_vs_direct": float((uf - u).abs().max() / u.abs().max())}}


# ---------------------------------------------------------------- our arm
def ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_1708_09162_gb300 import build
    build.build()
    from paper_1708_09162_gb300 import ibem

    oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.operator_only and not args.fp32_only \
            and not (args.batch_only or args.learned_only or args.cnn_forward_only or args.laplace_only
                     or args.learned_config5 or args.fmm_error_study or args.config4):
        oracle = start_oracle_child()             # CPU only; overlaps the GPU setup below
    torch.cuda.set_device(local_rank)
    dist = world > 1
    if dist:
        import torch.distributed as td

    def barrier():
        if dist:
            td.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.Stream()
    if args.batch_only:
        print(json.dumps({"batched_instances": batched_instances(ibem, stream, args)}), flush=True)
        return
    if args.cnn_forward_only:
        c = ibem.ibem_cnn_create(32, seed=SEED, stream=stream)
        out = cnn_forward_timing(ibem, stream, c)
        ibem.ibem_cnn_destroy(c)
        print(json.dumps({"cnn_forward": out}), flush=True)
        return
    if args.learned_only:
        print(json.dumps({"learned_preconditioner": learned_preconditioner(ibem, stream, args)}), flush=True)
        return
    if args.learned_config5:
        print(json.dumps({"learned_config5": learned_config5(ibem, stream, args)}), flush=True)
        return
    if args.fmm_error_study:
        print(json.dumps({"fmm_error_study": fmm_error_study(ibem, stream, args)}), flush=True)
        return
    if args.config4:
        print(json.dumps({"config4": config4_section(ibem, stream, args)}), flush=True)
        return
    if args.laplace_only:
        print(json.dumps({"laplace": laplace_section(ibem, stream, world, barrier, args.steps, args.warmup)}),
              flush=True)
        return

    W = WORKLOAD
    R = W["nrhs"]
    t0 = time.perf_counter()
    h = ibem.ibem_create(ibem.sphere_patches(), ibem.make_params(
        W["p"], W["m"], q_cheb=W["q_cheb"], eta=W["eta"], kernel=ibem.IBEM_HELMHOLTZ, kappa=W["kappa"],
        fp64_coupling=ibem.IBEM_COUPLING_SLICED if args.coupling == "sliced" else ibem.IBEM_COUPLING_GENERATE),
        stream)
    t_create = time.perf_counter() - t0
    t0 = time.perf_counter()
    ibem.ibem_assemble(h)
    t_assemble = time.perf_counter() - t0
    info = ibem.ibem_get_info(h)
    N = info.ndof
    b = plane_wave_rhs(ibem, h, W["kappa"], R, SEED + 3)           # [R][N][2]: the 64 plane waves
    y = torch.empty_like(b)
    y32 = torch.empty_like(b)

    def run(steps, precision, out):
        with torch.cuda.stream(stream):
            for _ in range(steps):
                ibem.ibem_matvec(h, b, out, R, precision)

    if args.fp32_only:
        if args.fp32_store:
            ibem.ibem_set_fp32_coupling(h, ibem.IBEM_FP32_COUPLING_STORE)
        run(max(1, args.warmup), 1, y32)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        run(args.steps, 1, y32)
        ev1.record(stream)
        barrier()
        print(json.dumps({"fp32_ms": ev0.elapsed_time(ev1) / args.steps,
                          "stored_ring_depth": ibem.ibem_get_info(h).stored_ring_depth}), flush=True)
        return
    oracle_res = finish_oracle_child(*oracle) if oracle else None

    # ---- headline: FP64-accurate operator, 64 right-hand sides ----
    run(args.warmup, 0, y)
    ibem.ibem_profile_read(h)
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ibem.ibem_profile_enable(h, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    run(args.steps, 0, y)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = ibem.ibem_profile_read(h)
    ibem.ibem_profile_enable(h, False)
    clk = clocks.stop()
    ms = max_over_ranks(ms)
    value = job_throughput(world, N * R, ms * 1e-3)
    phase_ms = {k: v / args.steps for k, v in prof["ms"].items()}

    # ---- roofline of the dominant kernel (the coupling; FP32 pipe) ----
    _, sm_max, peak_src = _peaks()
    alu_peak = 152 * 128 * sm_max * 1e6 / 1e12                      # FP32 lane operations per second (T)
    coup_ms = phase_ms["coupling"]
    kvals = info.n_far * float(W["q_cheb"]) ** 4
    if args.coupling == "sliced":
        ops, tflop = sliced_ops_per_launch(info.n_far, R)
        tpk0, _ = _peak_tensor()
        achieved = ops / (coup_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s", "frac": achieved / alu_peak,
                "traffic": _profile_traffic(), "kernel": "helm_coupling_sliced_kernel", "ms_per_launch": coup_ms,
                "algorithmic_ops": ops, "kernel_values": kvals, "kernel_values_per_s": kvals / (coup_ms * 1e-3),
                "tensor": {"flops": tflop, "achieved_tflops": tflop / (coup_ms * 1e-3) / 1e12, "peak_tflops": tpk0,
                           "frac": tflop / (coup_ms * 1e-3) / 1e12 / tpk0},
                "peak_source": "FP32 pipe: 152 SMs x 128 lanes x %.0f MHz (sm_max_mhz of MEASURED_PEAKS.json, %s)"
                               % (sm_max, peak_src),
                "ops_source": "counted from the digit-sliced formulas per far block and chunk of 32 right-hand sides: "
                              "247 FP32 operations per generated complex kernel value, 58 per sliced real value, "
                              "48 per recombined accumulator entry; tensor: 21 slice pairs of 2 x 128 x 64 x 64"}
    else:
        gen_ops, mac_ops = gen_ops_per_launch(info.n_far, W["q_cheb"], R)
        achieved = (gen_ops + mac_ops) / (coup_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s", "frac": achieved / alu_peak,
                "traffic": _profile_traffic(), "kernel": "helm_coupling_gen_kernel", "ms_per_launch": coup_ms,
                "algorithmic_ops": gen_ops + mac_ops, "ops_generation": gen_ops, "ops_multiply_add": mac_ops,
                "kernel_values": kvals, "kernel_values_per_s": kvals / (coup_ms * 1e-3),
                "peak_source": "FP32 pipe: 152 SMs x 128 lanes x %.0f MHz (sm_max_mhz of MEASURED_PEAKS.json, %s)"
                               % (sm_max, peak_src),
                "ops_source": "counted from the double-float formulas: 247 FP32 operations per generated complex "
                              "kernel value, 48 per complex multiply-add and right-hand side"}

    # ---- FP32 operator (tensor-core coupling, BF16 K and moments) ----
    run(args.warmup, 1, y32)
    barrier()
    ibem.ibem_profile_enable(h, True)
    ev0.record(stream)
    run(args.steps, 1, y32)
    ev1.record(stream)
    barrier()
    ms32 = ev0.elapsed_time(ev1) / args.steps
    p32 = ibem.ibem_profile_read(h)
    ibem.ibem_profile_enable(h, False)
    c32 = p32["ms"]["coupling"] / args.steps
    err32 = float((y32 - y).abs().max() / y.abs().max())
    flops_tc = 2.0 * 128 * 128 * R * info.n_far                      # real-form GEMM per far block
    tpk, tsrc = _peak_tensor()
    fp32 = {"value": world * N * R / (ms32 * 1e-3), "ms_per_step": ms32, "coupling_ms": c32,
            "rel_err_vs_fp64_all_64": err32,
            "tensor": {"kernel": "mr_coupling_tc_kernel", "achieved_tflops": flops_tc / (c32 * 1e-3) / 1e12,
                       "peak_tflops": tpk, "frac": flops_tc / (c32 * 1e-3) / 1e12 / tpk,
                       "peak_source": "MEASURED_PEAKS.json bf16_tflops (%s)" % tsrc}}

    # ---- the same operator with the coupling stored in BF16 at assembly ----
    fp32_stored = None
    if not args.no_store:
        t0 = time.perf_counter()
        st_status = ibem.ibem_set_fp32_coupling_status(h, ibem.IBEM_FP32_COUPLING_STORE)
        t_store = time.perf_counter() - t0
        fp32_stored = {"status": ibem.ibem_status_string(st_status), "store_s": t_store}
        if st_status == 0:
            y32s = torch.empty_like(b)
            run(args.warmup, 1, y32s)
            barrier()
            ibem.ibem_profile_enable(h, True)
            ev0.record(stream)
            run(args.steps, 1, y32s)
            ev1.record(stream)
            barrier()
            ms32s = ev0.elapsed_time(ev1) / args.steps
            p32s = ibem.ibem_profile_read(h)
            ibem.ibem_profile_enable(h, False)
            c32s = p32s["ms"]["coupling"] / args.steps
            kbytes = info.n_far * 128 * 64 * 2                        # [Kr; Ki] BF16 per far block
            mbytes = info.n_clusters * 2 * R * 64 * 2                 # BF16 moments of every cluster, once
            xbytes = info.n_far * 2 * R * 64 * 2                      # the same, requested once per far block
            hbm, _, hsrc = _peaks()
            fp32_stored.update({
                "value": world * N * R / (ms32s * 1e-3), "ms_per_step": ms32s, "coupling_ms": c32s,
                "rel_err_vs_fp64_all_64": float((y32s - y).abs().max() / y.abs().max()),
                "max_diff_vs_generated": float((y32s - y32).abs().max() / y32.abs().max()),
                "stored_gb": kbytes / 1e9,
                "ring_depth": ibem.ibem_get_info(h).stored_ring_depth,
                "tensor": {"kernel": "mr_coupling_stored_kernel",
                           "achieved_tflops": flops_tc / (c32s * 1e-3) / 1e12, "peak_tflops": tpk,
                           "frac": flops_tc / (c32s * 1e-3) / 1e12 / tpk,
                           "peak_source": "MEASURED_PEAKS.json bf16_tflops (%s)" % tsrc},
                "hbm": {"bytes_per_launch": kbytes + mbytes, "moment_bytes_requested": xbytes,
                        "achieved_gbs": (kbytes + mbytes) / (c32s * 1e-3) / 1e9, "peak_gbs": hbm,
                        "frac": (kbytes + mbytes) / (c32s * 1e-3) / 1e9 / hbm,
                        "note": "algorithmic HBM bytes = the stored blocks and every cluster's BF16 moments, "
                                "each read once; the moments are requested once per far block and served "
                                "from L2 where neighbouring target rows share source clusters"}})
            del y32s

    # ---- both operators against the oracle on sampled rows at full size ----
    accuracy = None
    if oracle_res is not None:
        rows, xs = sampled_input(N)
        X = np.zeros((16, N), dtype=complex)
        X[0] = xs
        X[1:] = np.random.default_rng(SEED + 12).normal(size=(15, N))
        xd = torch.from_numpy(np.ascontiguousarray(np.stack([X.real, X.imag], -1))).cuda()
        yd = torch.empty_like(xd)
        yo = np.array(oracle_res["y"])
        yo = yo[:, 0] + 1j * yo[:, 1]
        accuracy = {"rows": len(rows), "rhs": "one seeded complex normal vector (column 0 of a 16-column block)"}
        for name, prec in (("fp64", 0), ("fp32_tensor_core", 1)):
            ibem.ibem_matvec(h, xd, yd, 16, prec)
            torch.cuda.synchronize()
            yy = yd[0].cpu().numpy()
            yy = (yy[:, 0] + 1j * yy[:, 1])[rows]
            accuracy[name] = float(np.max(np.abs(yy - yo)) / np.max(np.abs(yo)))

    # ---- end to end through the host-buffer entry point ----
    bh = torch.empty((R, N, 2), dtype=torch.float64, pin_memory=True)
    bh.copy_(b.cpu())
    yh = torch.empty((R, N, 2), dtype=torch.float64, pin_memory=True)
    e2e_steps = max(2, args.steps // 5)
    ibem.ibem_matvec_host(h, bh, yh, R)
    barrier()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        ibem.ibem_matvec_host(h, bh, yh, R)
    e2e_s = max_over_ranks((time.perf_counter() - t) / e2e_steps)

    # ---- lock-step GMRES of the plane waves to true relative residual 1e-8 ----
    solve = None
    if not args.no_solve and not args.operator_only:
        solve = {"rtol": 1e-8, "precond": "block-Jacobi", "solver": "lock-step GMRES(100)"}

        def solve_once(nr, prec):
            w = torch.empty_like(b[:nr])
            s, si = ibem.ibem_solve(h, b[:nr].contiguous(), w, nr, rtol=1e-8, maxit=5000,
                                    precond=ibem.IBEM_PRECOND_BLOCK_JACOBI, precision=prec, check=False)
            return {"status": ibem.ibem_status_string(s), "seconds": si.seconds, "steps": si.steps,
                    "iterations": si.iterations, "outer": si.outer, "rel_residual_fp64": si.rel_residual}

        solve["mixed_64"] = solve_once(R, 1)
        solve["mixed_16"] = solve_once(16, 1)
        if not args.no_fp64_solve:
            solve["fp64_16"] = solve_once(16, 0)
            solve["speedup_mixed_vs_fp64_16rhs"] = solve["fp64_16"]["seconds"] / solve["mixed_16"]["seconds"]

    pot = None if (args.no_potential or args.operator_only) else potentials_section(ibem, stream, h, b)
    ibem.ibem_destroy(h)

    lap = None if (args.no_laplace or args.operator_only) else laplace_section(
        ibem, stream, world, barrier, max(10, args.steps), args.warmup)
    batched = None if (args.no_batch or args.operator_only) else batched_instances(ibem, stream, args)
    learned = None if (args.no_learned or args.operator_only) else learned_preconditioner(ibem, stream, args)

    cpu = None
    if oracle_res is not None:
        cpu = {"value": len(oracle_res["rows"]) / oracle_res["seconds"], "unit": UNIT, "cores": oracle_res["workers"],
               "cpu": oracle_res["cpu"], "host_cores": oracle_res["cores"], "kind": "oracle",
               "sample": "%d rows of the oracle's FMM-mode operator of the same workload applied to one right-hand "
                         "side, one forked worker per core (near blocks and the moments the rows use included; "
                         "the operator's tree, built once in %.0f s, excluded)"
                         % (len(oracle_res["rows"]), oracle_res["setup_s"])}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("f64 (coupling in BF16 digit slices on tcgen05 with exact FP32 accumulation and double-float "
                      "recombination, about 45 bits; FP64 near field)" if args.coupling == "sliced" else
                      "f64 (double-float coupling, about 48 bits; FP64 near field)"),
            "data": "synthetic",
            "config": dict(W, ndof=N, ndof_super=info.ndof_super, n_near=info.n_near, n_far=info.n_far,
                           parallelism="replicas" if world > 1 else "single",
                           l2="inputs larger than L2: %.1f GB of FP64 near blocks and %.1f GB of moments read "
                              "per step" % (info.bytes_near / 1e9, info.n_far * 64 * R * 16 / 1e9)),
            "phase_ms": phase_ms, "create_s": t_create, "assemble_s": t_assemble,
            "roofline": roof,
            "fp32_tensor_core": fp32,
            "fp32_tensor_core_stored": fp32_stored,
            "accuracy_vs_oracle_rows": accuracy,
            "solve": solve,
            "potential": pot,
            "laplace_p3_m5": lap,
            "batched_instances": batched,
            "learned_preconditioner": learned,
            "cpu_baseline": cpu,
            "e2e": {"value": world * N * R / e2e_s, "unit": UNIT, "h2d_bytes_per_step": N * R * 16,
                    "d2h_bytes_per_step": N * R * 16},
            "gpu_launches": prof["launches"],
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.oracle_child:
        oracle_child(args.oracle_child)
        return
    if args.m is not None:
        WORKLOAD["m"] = args.m
        WORKLOAD["workload"] = "helmholtz-sphere-p2-m%d-q8-k4-R64" % args.m
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
