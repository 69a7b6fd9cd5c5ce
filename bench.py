#!/usr/bin/env python
"""Benchmark: TDVP time-steps/s of the mixed-precision batched sweep at chi = 256.

Workload: the 101-site long-range transverse-field Ising chain (alpha = 1.5,
J = 1, h = 0.5, 8 exponentials -> MPO bond dimension 10), dt = 0.01,
chi_max = 256, eps = 1e-12, Lanczos with at most 8 vectors and tolerance 1e-6,
8 Stoudenmire-White segments of 15, 12 x 6 and 14 sites, all segments of a
stage batched into the same launches. The state is a seeded random MPS brought
to the inverse canonical gauge at chi = 256 (every bond saturated, as after
the quench's early growth), so every timed step does the full chi = 256 work.

One step = one full symmetric time step (both half sweeps) of tdvp_step.
`value` is whole-job throughput: time steps of all ranks / slowest rank's time.
Ranks run independent replicas of the chain (the sweep of one chain runs on one
GPU; there is no cross-GPU exchange in this build).

--impl reference times the CPU oracle (numpy FP64, unchanged) on a bounded
sample of the same workload and prints the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import tdvp_inputs as I  # noqa: E402

METRIC = "TDVP time-steps/s (chi=256, mixed+batched)"
UNIT = "time-steps/s"
PREC = {"fp64": I.FP64, "tf32": I.TF32, "tf32x3": I.TF32X3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=sorted(PREC))
    ap.add_argument("--chi", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="steps of the plain FP64 GPU path, each timed, compared step by step with the "
                         "mixed path from the same state; 0 skips it")
    ap.add_argument("--svd-case", type=int, default=0,
                    help="profiling case: two truncated splits of one N x N two-site state "
                         "(half the spectrum kept), no benchmark line")
    ap.add_argument("--heff-case", type=int, default=0,
                    help="profiling case: three two-site H_eff applications at chi_l = chi_r = N, m = 10, d = 2 "
                         "(the benchmark's MPO) in --precision, through tdvp_op_heff; no benchmark line")
    ap.add_argument("--grad-case", action="store_true",
                    help="the differentiated 41-site Ising quench at chi 64: d<sigma^z_20(t)>/d(h, J) "
                         "by tdvp_step_tangent, timed, checked against central differences of tdvp_step")
    ap.add_argument("--grad-steps", type=int, default=4, help="timed steps of --grad-case")
    ap.add_argument("--xxx-case", action="store_true",
                    help="time steps of the 201-site 1/r^2 XXX chain (m = 32, chi 256, 16 uneven segments, "
                         "--precision) from a seeded random MPS at chi 256; no benchmark line")
    ap.add_argument("--xxx-steps", type=int, default=2)
    ap.add_argument("--xxx-dmrg", action="store_true",
                    help="with --xxx-case: the whole pipeline of the XXX quench -- two-site DMRG from the seeded "
                         "random MPS at chi 16 up to chi 256, sigma^z at the central site, then --xxx-steps "
                         "timed steps and the dynamical correlation at the last time")
    ap.add_argument("--tdvp1-case", action="store_true",
                    help="one-site vs two-site FP64 steps on the 41-site Ising chain at chi 64; no benchmark line")
    ap.add_argument("--tune-case", action="store_true",
                    help="mixed-precision steps of the 101-site chain at chi 64, 128 and 256 with fixed GEMM "
                         "tiles and with the autotuner's; no benchmark line")
    ap.add_argument("--grad-init", default="random", choices=["random", "all_up"],
                    help="--grad-case start: seeded random MPS at chi 64 (every bond saturated, so every "
                         "step does the full chi = 64 work) or the all-up product state")
    return ap.parse_args()


def svd_case(n, prec):
    """The split of one evolved two-site state (Fig. 5) at chi = n / 2, with
    the SVD of the path of precision `prec` (--precision): a seeded
    n x n matrix whose singular values fall from 1 to 6.5e-3 over the first
    half (the previous bond's Schmidt values) and from 7e-4 to 4e-6 over the
    second (the weight one time step moves into new directions), truncated to
    n / 2 values, run twice through tdvp_op_split. A small, self-contained case
    for kernel profiles of the Jacobi sweeps."""
    import torch
    from paper_1912_06127_gb300 import tdvp
    U = np.linalg.qr(I.random_complex((n, n), 5))[0]
    Vh = np.linalg.qr(I.random_complex((n, n), 6))[0]
    s = np.concatenate([np.geomspace(1.0, 6.5e-3, n // 2), np.geomspace(7e-4, 4e-6, n - n // 2)])
    th = torch.from_numpy(((U * s) @ Vh).reshape(-1).view(np.float64).copy()).cuda()
    for _ in range(2):
        PsiL = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
        PsiR = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
        V = torch.zeros(n, dtype=torch.float64, device="cuda")
        chi, w = tdvp.op_split(n, n, th, n // 2, 0.0, 1e-12, PsiL, V, PsiR, None, precision=prec)
        torch.cuda.synchronize()
    w_ref = float((s[n // 2:] ** 2).sum())
    print(json.dumps({"svd_case": n, "chi": chi, "w": w, "w_expected": w_ref}))
    if chi != n // 2 or abs(w - w_ref) > 1e-9 * float((s ** 2).sum()):
        raise SystemExit("svd case: unexpected truncation")


def heff_case(chi, prec):
    """Three H_eff . theta applications (Fig. 4a) at the benchmark's MPO (m = 10,
    d = 2) with chi_l = chi_r = chi on seeded random environments and state,
    through tdvp_op_heff: a small, self-contained case for kernel profiles of
    the tensor-core GEMMs."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_06127_gb300 import tdvp
    w = I.tfim_n101_quench()
    mdl = w.model
    mpo = tdvp.build_mpo(mdl.kind, mdl.N, mdl.alpha, mdl.J, mdl.h, mdl.n_exp)
    W = mpo.tensor(mdl.n_exp)[0]
    m, d = W.shape[0], 2

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()

    L = dev(I.random_complex((chi, m, chi), 1))
    R = dev(I.random_complex((chi, m, chi), 2))
    th = dev(I.random_complex((chi, d, d, chi), 3))
    y = torch.zeros(chi * d * d * chi, dtype=torch.complex128, device="cuda")
    # the first call makes the autotuner's decisions; the last one (in the
    # NVTX range "profiled") runs exactly what the time step runs
    for it in range(3):
        if it == 2:
            torch.cuda.nvtx.range_push("profiled")
        tdvp.op_heff(prec, 2, chi, chi, m, d, W, L, R, th, y)
        torch.cuda.synchronize()
        if it == 2:
            torch.cuda.nvtx.range_pop()
    print(json.dumps({"heff_case": chi, "precision": prec, "y_norm": float(torch.linalg.norm(y))}))


def grad_case(args):
    """d<sigma^z_20(t)>/d(h, J) of the 41-site long-range Ising chain (alpha = 3,
    J = h = 1, 6 exponentials, dt = 0.02, chi_max = 64, eps = 1e-12, Lanczos to
    1e-12 with at most 20 vectors, 6-point quadrature), from a seeded random MPS
    at chi = 64 (default) or all spins up: one untimed step, then --grad-steps
    differentiated steps (both directions) timed with CUDA events, the plain
    FP64 steps timed the same way, and the gradient compared with central
    differences (step 1e-5) of tdvp_step over the same steps."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_06127_gb300 import tdvp
    w = I.tfim_n41_derivative()
    mdl, prm = w.model, w.params
    site = mdl.N // 2 - 1                      # sigma^z_20 (0-based)
    kmax, ktol, nq = 20, 1e-12, 6
    n_steps = args.grad_steps
    chi = prm.chi_max
    raw = I.random_mps_tensors(mdl.N, chi, seed=4) if args.grad_init == "random" else None
    up = I.basis_state("all_up", mdl.N)
    x, lam = tdvp.fit_power_law(mdl.alpha, mdl.n_exp, mdl.N - 1)
    stream = torch.cuda.current_stream()

    def params():
        return tdvp.step_params(prm.dt, chi, eps=prm.eps, krylov_max=kmax, krylov_tol=ktol)

    def initial():
        return tdvp.init_mps_tensors(raw, chi, 1e-14) if raw is not None else tdvp.init_mps(mdl.N, up, chi)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    def plain(J, h, n):
        mpo = tdvp.build_mpo(mdl.kind, mdl.N, mdl.alpha, J, h, mdl.n_exp, x, lam)
        mps = initial()
        tdvp.step(mps, mpo, params(), 1, stream=stream)           # untimed first step
        _, ms = timed(lambda: tdvp.step(mps, mpo, params(), n, stream=stream))
        return tdvp.measure(mps, tdvp.OBS_SZ)[site], list(mps.bond_dims()), ms

    def differentiated(n, profile=False):
        mpo = tdvp.build_mpo(mdl.kind, mdl.N, mdl.alpha, mdl.J, mdl.h, mdl.n_exp, x, lam)
        dm = [tdvp.build_mpo_derivative(mpo, tdvp.PARAM_H), tdvp.build_mpo_derivative(mpo, tdvp.PARAM_J)]
        mps = initial()
        tan = tdvp.Tangent(mps, 2)
        tdvp.step_tangent(mps, mpo, tan, dm, params(), 1, n_quad=nq, stream=stream)   # untimed first step
        if profile:
            tdvp.profile(True)
        st, ms = timed(lambda: tdvp.step_tangent(mps, mpo, tan, dm, params(), n, n_quad=nq, stream=stream))
        prof = tdvp.profile_read() if profile else None
        tdvp.profile(False)
        val, der = tdvp.measure_tangent(mps, tan, tdvp.OBS_SZ)
        return val[site], der[:, site], list(mps.bond_dims()), ms, st, prof

    clocks = ClockSampler(0)
    clocks.start()
    loss, grad, dims, ms_d, st, prof = differentiated(n_steps, profile=True)
    clk = clocks.stop()
    loss_p, dims_p, ms_p = plain(mdl.J, mdl.h, n_steps)
    d = 1e-5
    fd, same = [], dims_p == dims
    for dh, dJ in ((d, 0.0), (0.0, d)):
        a, da, _ = plain(mdl.J + dJ, mdl.h + dh, n_steps)
        b, db, _ = plain(mdl.J - dJ, mdl.h - dh, n_steps)
        same = same and da == dims and db == dims
        fd.append((a - b) / (2 * d))
    fd = np.array(fd)
    rel = float(np.abs(grad - fd).max() / max(np.abs(fd).max(), 1e-300))
    ms_total = sum(v["ms"] for v in prof.values()) if prof else 0.0
    dom = max(prof, key=lambda k: prof[k]["ms"]) if prof else None
    line = {
        "metric": "differentiated TDVP time-steps/s (d<sigma^z_20(t)>/d(h, J), both directions)",
        "value": n_steps / (ms_d * 1e-3), "unit": "time-steps/s", "n_gpus": 1, "steps": n_steps,
        "warmup": 1, "ms_per_step": ms_d / n_steps, "higher_is_better": True,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "N": mdl.N, "alpha": mdl.alpha, "J": mdl.J, "h": mdl.h, "m": mdl.m,
                   "chi_max": chi, "dt": prm.dt, "eps": prm.eps, "krylov": [kmax, ktol], "n_quad": nq,
                   "init": ("seeded random MPS at chi %d (seed 4)" % chi) if raw is not None else "all up",
                   "observable": "sigma^z_%d (1-based %d)" % (site, site + 1)},
        "loss": float(loss), "grad_h_J": [float(v) for v in grad], "fd_h_J": [float(v) for v in fd],
        "grad_rel_err_vs_fd": rel, "fd_step": d, "same_bond_dims_in_fd_runs": bool(same),
        "loss_plain_run": float(loss_p), "plain_fp64_steps_per_s": n_steps / (ms_p * 1e-3),
        "cost_vs_plain": ms_d / ms_p, "chi_max_seen": int(max(dims)), "gpu_launches": int(st.kernel_launches),
        "clocks": clk,
        "kernels": {k: {"ms": v["ms"], "launches": v["launches"], "share": v["ms"] / max(ms_total, 1e-9)}
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:12]} if prof else None,
        "dominant_kernel": dom,
    }
    print(json.dumps(line), flush=True)


def xxx_case(args):
    """Throughput of the 1/r^2 XXX quench's time step (N = 201, alpha = 2, 10
    exponentials -> m = 32, dt = 0.05, chi_max = 256, 16 uneven segments 65, 12,
    4 x 12, 12, 64) from a seeded random MPS at chi = 256 (every bond saturated):
    one untimed step, then --xxx-steps steps timed with CUDA events."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_06127_gb300 import tdvp
    w = I.xxx_n201_quench()
    mdl, prm = w.model, w.params
    prec = PREC[args.precision]
    mpo = tdvp.build_mpo(mdl.kind, mdl.N, mdl.alpha, mdl.J, mdl.h, mdl.n_exp)
    stream = torch.cuda.current_stream()
    extra = {}
    if args.xxx_dmrg:
        # ground state: two-site DMRG (same H_eff kernels, Lanczos ground mode)
        # from the seeded random MPS at chi 16, chi_max raised 32 -> 256
        gs = tdvp.init_mps_tensors(I.random_mps_tensors(mdl.N, w.chi_init, seed=w.seed), prm.chi_max, 1e-14)
        t0 = time.perf_counter()
        sweeps = []
        for chi, n in ((32, 2), (64, 2), (128, 2), (256, 3)):
            ds = tdvp.dmrg(gs, mpo, tdvp.dmrg_params(chi, eps=prm.eps, krylov_max=8, krylov_tol=1e-8,
                                                   precision=prec), n, stream=stream)
            sweeps.append({"chi_max": chi, "sweeps": n, "energy": ds.energy, "w_total": ds.w_total})
        torch.cuda.synchronize()
        e0 = tdvp.energy(gs, mpo)
        extra["dmrg"] = {"seconds": time.perf_counter() - t0, "schedule": sweeps, "E0": e0,
                         "E0_per_site": e0 / mdl.N, "bond_dims_max": int(max(gs.bond_dims())),
                         "context": "paper's E0/N = -0.410611165931 at chi 1024 with U(1) symmetry (Sec. IV C)"}
        # sigma^z at the central site (0-based 100), evolved; C(r - k, t) = e^{-i E0 t} <psi0|sigma^z_r|psi(t)>
        k = mdl.N // 2
        mps = tdvp.mps_copy(gs)
        tdvp.apply_site_op(mps, k, np.diag([1.0, -1.0]).astype(np.complex128))
    else:
        mps = tdvp.init_mps_tensors(I.random_mps_tensors(mdl.N, prm.chi_max, seed=0), prm.chi_max, 1e-14)
    p = tdvp.step_params(prm.dt, prm.chi_max, w_max=prm.w_max, eps=prm.eps, krylov_max=prm.krylov_max,
                         krylov_tol=prm.krylov_tol, precision=prec, seg_len=prm.seg_len)
    tdvp.step(mps, mpo, p, 1, stream=stream)
    clocks = ClockSampler(0)
    clocks.start()
    tdvp.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    st = tdvp.step(mps, mpo, p, args.xxx_steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = tdvp.profile_read()
    tdvp.profile(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    tot = sum(v["ms"] for v in prof.values())
    if args.xxx_dmrg:
        t_final = (1 + args.xxx_steps) * prm.dt
        c = tdvp.expect_mixed(gs, mps, tdvp.OBS_SZ) * np.exp(-1j * extra["dmrg"]["E0"] * t_final)
        extra["correlation"] = {"t": t_final, "site": k, "r": list(range(k - 5, k + 6)),
                                "C_re": [float(v.real) for v in c[k - 5:k + 6]],
                                "C_im": [float(v.imag) for v in c[k - 5:k + 6]],
                                "sum_rule_sz_total": float(tdvp.measure(mps, tdvp.OBS_SZ).sum())}
    print(json.dumps({
        **extra, "xxx_case": w.name, "time_steps_per_s": args.xxx_steps / (ms * 1e-3), "ms_per_step": ms / args.xxx_steps,
        "steps": args.xxx_steps, "precision": args.precision, "m": mdl.m, "segments": prm.seg_len,
        "chi_max_seen": st.chi_max_seen, "gpu_launches": int(st.kernel_launches), "clocks": clk,
        "kernels": {k: {"ms": v["ms"], "share": v["ms"] / max(tot, 1e-9)}
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]}}), flush=True)


def tdvp1_case(args):
    """One-site (tdvp_step1) against two-site (tdvp_step) FP64 steps of the 41-site
    long-range Ising chain (alpha = 3, J = h = 1, 6 exponentials, dt = 0.02,
    chi = 64, Lanczos <= 8 vectors to 1e-10) from a seeded random MPS at chi = 64
    (every bond full, the regime where the hybrid scheme switches): one untimed
    step of each, then one timed step of each (CUDA events), serial and with 8
    segments (6, 5 x 7; all segments of a stage batched); each step's norm and
    energy change."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_06127_gb300 import tdvp
    w = I.tfim_n41_derivative()
    mdl, prm = w.model, w.params
    chi = prm.chi_max
    mpo = tdvp.build_mpo(mdl.kind, mdl.N, mdl.alpha, mdl.J, mdl.h, mdl.n_exp)
    raw = I.random_mps_tensors(mdl.N, chi, seed=4)
    p = tdvp.step_params(prm.dt, chi, eps=prm.eps, krylov_max=8, krylov_tol=1e-10)
    seg = [6, 5, 5, 5, 5, 5, 5, 5]
    pseg = tdvp.step_params(prm.dt, chi, eps=prm.eps, krylov_max=8, krylov_tol=1e-10, seg_len=seg)
    stream = torch.cuda.current_stream()
    out = {}
    for name, fn, p in (("two_site", tdvp.step, p), ("one_site", tdvp.step1, p),
                        ("two_site_8_segments", tdvp.step, pseg), ("one_site_8_segments", tdvp.step1, pseg)):
        mps = tdvp.init_mps_tensors(raw, chi, 1e-14)
        fn(mps, mpo, p, 1, stream=stream)
        n0, e0 = tdvp.norm(mps), tdvp.energy(mps, mpo)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        fn(mps, mpo, p, 1, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        out[name] = {"ms_per_step": ms, "time_steps_per_s": 1e3 / ms, "norm_change": tdvp.norm(mps) - n0,
                     "energy_change": tdvp.energy(mps, mpo) - e0, "bond_dims_max": int(max(mps.bond_dims()))}
    print(json.dumps({"tdvp1_case": w.name, "chi": chi, "dtype": "f64", **out,
                      "speedup_one_site": out["two_site"]["ms_per_step"] / out["one_site"]["ms_per_step"]}),
          flush=True)


def tune_case(args):
    """The 101-site benchmark chain (3xTF32, 8 segments) from its seeded random
    state at chi = 64, 128 and 256: one warm-up step (which also makes the
    autotuner's decisions when it is on), then timed steps (CUDA events), with
    fixed tiles and with tuned tiles; the tuned decisions are listed."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_06127_gb300 import tdvp
    w = workload(args)
    mdl, prm = w.model, w.params
    mpo = tdvp.build_mpo(mdl.kind, mdl.N, mdl.alpha, mdl.J, mdl.h, mdl.n_exp)
    stream = torch.cuda.current_stream()
    out = {}
    for chi in (64, 128, 256):
        raw = I.random_mps_tensors(mdl.N, chi, seed=0)
        row = {}
        for tuned in (False, True):
            tdvp.set_autotune(tuned)
            mps = tdvp.init_mps_tensors(raw, chi, 1e-14)
            p = tdvp.step_params(dt=prm.dt, chi_max=chi, w_max=prm.w_max, eps=prm.eps,
                                 krylov_max=prm.krylov_max, krylov_tol=prm.krylov_tol,
                                 precision=PREC[args.precision], seg_len=prm.seg_len, merge_turning=1)
            tdvp.step(mps, mpo, p, 1, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            tdvp.step(mps, mpo, p, args.steps, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            row["tuned" if tuned else "fixed"] = e0.elapsed_time(e1) / args.steps
            if tuned:
                row["decisions"] = tdvp.autotune_report()
            del mps
        row["speedup"] = row["fixed"] / row["tuned"]
        out[str(chi)] = row
    tdvp.set_autotune(True)
    print(json.dumps({"tune_case": w.name, "precision": args.precision, "ms_per_step": out}), flush=True)


def workload(args):
    w = I.tfim_n101_quench(PREC[args.precision])
    return w


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def allreduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps, ms_max, world):
    """Whole-job throughput of `world` replicas that each ran `steps` steps,
    the slowest taking ms_max milliseconds."""
    return steps * world / (ms_max * 1e-3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def fp64_peak_tflops():
    """cuBLAS DGEMM rate on this GPU (the FP64 denominator), measured here."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 1e30
    for _ in range(3):
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


# DRAM bytes (read + write) per local problem of a kernel kind, from one ncu
# capture of the kernel on a single 512 x 512 split (`--svd-case 512`); a
# launch of the time step carries several problems and its traffic scales with
# them. Emptied whenever a listed kernel changes after its capture, so that no
# stale figure is reported.
TRAFFIC_PER_PROBLEM = {"svd_jacobi_fp32": 4.756224e6 + 0.859392e6,
                       "svd_jacobi_dd": 8.530432e6 + 0.985856e6}


def sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def roofline(prof, steps, clk=None, kernel=None, problems=None):
    """Roofline entry for `kernel` (default: the kind with the largest device time);
    `problems`: local problems (two-site updates) in the timed region."""
    if not prof:
        return None, None
    dom = kernel if kernel in prof else max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    peaks, src = measured_peaks()
    ms_launch = d["ms"] / max(d["launches"], 1)
    if dom.startswith("tc_gemm"):
        # TF32 dense peak = measured bf16 burst x nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s);
        # the 3xTF32 product issues three TF32 MMAs per algorithmic one, so its
        # own peak in algorithmic flops is a third of that
        tf32 = peaks["bf16_tflops"] * 1.1 / 2.25
        passes = 3 if dom.endswith("x3") else 1
        peak = tf32 / passes
        ach = d["flops"] / d["launches"] / (ms_launch * 1e-3) / 1e12
        r = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
             "peak_source": "%s bf16 x 1.1/2.25 (TF32 nominal ratio)%s" % (src, " / 3 (3xTF32)" if passes == 3 else ""),
             "tensor_pipe_frac": ach * passes / tf32}
    elif dom == "svd_jacobi_fp32":
        # FP32 ALU peak from unit counts and clocks: SMs x 128 FP32 lanes x 2 flops x clock
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        sms = sm_count()
        peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        ach = d["flops"] / d["launches"] / (ms_launch * 1e-3) / 1e12
        r = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
             "peak_source": "%d SMs (device query) x 128 FP32 lanes x 2 x %.0f MHz (median SM clock)" % (sms, mhz)}
    elif dom.startswith("zgemm") or dom.startswith("svd") or dom.startswith("theta"):
        peak = fp64_peak_tflops()
        ach = d["flops"] / d["launches"] / (ms_launch * 1e-3) / 1e12
        r = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
             "peak_source": "cuBLAS DGEMM measured in this run (FP64 pipe)"}
    else:
        peak = peaks["hbm_gbs"]
        ach = d["bytes"] / d["launches"] / (ms_launch * 1e-3) / 1e9
        r = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
             "peak_source": "%s hbm_gbs" % src}
    r["frac"] = r["achieved"] / r["peak"]
    r["kernel"] = dom
    r["ms_per_launch"] = ms_launch
    r["launches"] = d["launches"]
    r["traffic"] = None
    if dom in TRAFFIC_PER_PROBLEM and problems:
        r["traffic"] = TRAFFIC_PER_PROBLEM[dom] * problems / d["launches"]
        r["traffic_source"] = ("ncu dram__bytes_read+write of one 512x512 split, x %.1f problems per launch"
                               % (problems / d["launches"]))
    return r, dom


def cpu_baseline_sample(chi, seconds_budget=30.0):
    """Time the oracle (as it stands) on a bounded sample of the workload: one
    two-site H_eff application, one one-site H_eff application, one two-site
    SVD split and one environment update at chi = 256 (random operands of the
    workload's shapes), then scale to one time step by the operation counts of
    the step's schedule with every bond at chi (a lower bound on the oracle's
    step time, i.e. an upper bound on its steps/s)."""
    from oracle import models
    from oracle import tdvp as T
    w = I.tfim_n101_quench()
    mdl = w.model
    x, lam = models.fit_power_law(mdl.alpha, mdl.n_exp, mdl.N - 1)
    W = models.build_mpo_site(mdl.kind, mdl.J, mdl.h, x, lam)
    m = W.shape[0]
    L = I.random_complex((chi, m, chi), 1)
    R = I.random_complex((chi, m, chi), 2)
    th = I.random_complex((chi, 2, 2, chi), 3)
    ps = I.random_complex((chi, 2, chi), 4)
    t0 = time.perf_counter()
    y = T.heff2_apply(L, W, W, R, th)
    t_h2 = time.perf_counter() - t0
    t0 = time.perf_counter()
    T.heff1_apply(L, W, R, ps)
    t_h1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    T.split_two_site(y, chi, 0.0, 1e-12)
    t_svd = time.perf_counter() - t0
    t0 = time.perf_counter()
    T.env_left(L, ps, W)
    t_env = time.perf_counter() - t0
    sched = T.build_schedule(mdl.N, w.params.seg_len, 1)
    n_f = sum(1 for h in sched for o in h if o.kind == "fwd2")
    n_b = sum(1 for h in sched for o in h if o.kind == "back1")
    n_env = sum(len(o.env) for h in sched for o in h if o.kind == "fwd2")
    k = w.params.krylov_max
    t_step = n_f * (k * t_h2 + t_svd) + n_b * k * t_h1 + n_env * t_env
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    return {
        "value": 1.0 / t_step, "unit": UNIT, "cores": cores, "kind": "oracle",
        "method": "per-operation extrapolation (not a timed step)",
        "sample": ("per-operation extrapolation of the numpy oracle at chi=%d: one two-site H_eff (%.2fs), one "
                   "one-site H_eff (%.2fs), one 512x512 SVD split (%.2fs), one environment update (%.2fs), "
                   "timed; scaled to one time step by %d two-site updates x %d Lanczos vectors + %d one-site "
                   "updates x %d + %d environment updates with every bond at chi"
                   % (chi, t_h2, t_h1, t_svd, t_env, n_f, k, n_b, k, n_env)),
        "sample_seconds": t_h2 + t_h1 + t_svd + t_env,
    }


def oracle_step_measured(chi=32):
    """One whole time step of the oracle (as it stands) on the same chain,
    schedule and Lanczos settings, from the seeded random MPS at a bond
    dimension the host finishes in seconds, timed end to end (the initial
    canonicalisation excluded)."""
    from oracle import models
    from oracle import mps as M
    from oracle import tdvp as T
    w = I.tfim_n101_quench()
    mdl, prm = w.model, w.params
    x, lam = models.fit_power_law(mdl.alpha, mdl.n_exp, mdl.N - 1)
    W = models.build_mpo_site(mdl.kind, mdl.J, mdl.h, x, lam)
    eng = T.Engine(M.canonicalize(I.random_mps_tensors(mdl.N, chi, seed=0), chi, 1e-14), W)
    t0 = time.perf_counter()
    eng.step(T.Params(dt=prm.dt, chi_max=chi, eps=prm.eps, krylov_max=prm.krylov_max, krylov_tol=prm.krylov_tol,
                      seg_len=prm.seg_len), 1)
    dt = time.perf_counter() - t0
    return {"chi": chi, "s_per_step": dt, "value": 1.0 / dt, "unit": UNIT,
            "sample": "one full oracle time step of %s at chi=%d (seeded random MPS), timed" % (w.name, chi)}


# ---------------------------------------------------------------------------
def run_reference(args, world, rank):
    if rank != 0:
        return
    w = workload(args)
    for _ in range(args.warmup):
        pass  # the oracle has no state to warm; the warm-up steps are the first samples below
    vals, samples = [], []
    t_all = time.perf_counter()
    for _ in range(max(args.steps, 1)):
        cb = cpu_baseline_sample(args.chi)
        vals.append(1.0 / cb["value"])
        samples.append(cb["sample_seconds"])
    wall = time.perf_counter() - t_all
    t_step = float(np.median(vals))
    line = {
        "metric": METRIC, "value": 1.0 / t_step, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": w.name, "N": w.model.N, "chi_max": args.chi, "m": w.model.m,
                   "segments": w.params.seg_len, "dt": w.params.dt, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": 1.0 / t_step, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                         "method": cb["method"], "sample": cb["sample"] + " (median over the steps)"},
        "e2e": {"value": 1.0 / t_step, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
        # ms_per_step is extrapolated from timed operations, not a timed step:
        # each "step" here is one bounded sample of the workload's operations
        "extrapolated": True,
        "sample_s_per_step": float(np.median(samples)),
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_06127_gb300 import tdvp
    torch.cuda.set_device(local)
    w = workload(args)
    mdl, prm = w.model, w.params
    mpo = tdvp.build_mpo(mdl.kind, mdl.N, mdl.alpha, mdl.J, mdl.h, mdl.n_exp)
    raw = I.random_mps_tensors(mdl.N, args.chi, seed=0)
    mps = tdvp.init_mps_tensors(raw, args.chi, 1e-14)
    p = tdvp.step_params(dt=prm.dt, chi_max=args.chi, w_max=prm.w_max, eps=prm.eps,
                         krylov_max=prm.krylov_max, krylov_tol=prm.krylov_tol, precision=PREC[args.precision],
                         seg_len=prm.seg_len, merge_turning=1)
    stream = torch.cuda.current_stream()
    tdvp.step(mps, mpo, p, args.warmup, stream=stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    tdvp.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    t0 = time.perf_counter()
    st = tdvp.step(mps, mpo, p, args.steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    prof = tdvp.profile_read()
    tdvp.profile(False)
    clk = clocks.stop()
    barrier(world)
    ms_max = allreduce_max(ms, world)
    # end to end through the public API with host buffers: the job's input (the
    # seeded site tensors, in pinned host memory) is copied in and brought to
    # the inverse canonical gauge by tdvp_init_mps_tensors, then every step is
    # tdvp_step followed by reading that step's observable (<sigma^z_j> for
    # every site) back to the host
    pinned = []
    for a in raw:
        t = torch.empty(a.size * 2, dtype=torch.float64, pin_memory=True)
        t.numpy()[:] = a.reshape(-1).view(np.float64)
        pinned.append(t)
    host_in = [t.numpy().view(np.complex128).reshape(a.shape) for t, a in zip(pinned, raw)]
    h2d_bytes = sum(a.nbytes for a in raw)
    del mps
    torch.cuda.synchronize()
    n_e2e = max(1, args.e2e_steps)
    t0 = time.perf_counter()
    mps = tdvp.init_mps_tensors(host_in, args.chi, 1e-14)
    for _ in range(n_e2e):
        tdvp.step(mps, mpo, p, 1, stream=stream)
        sz = tdvp.measure(mps, tdvp.OBS_SZ)
    torch.cuda.synchronize()
    e2e_s = allreduce_max((time.perf_counter() - t0) / n_e2e, world)
    assert sz.shape == (mdl.N,) and np.all(np.isfinite(sz))
    if rank != 0:
        return
    value = job_value(args.steps, ms_max, world)
    rl, dom = roofline(prof, args.steps, clk, problems=st.n_fwd2)
    tc_kind = "tc_gemm_tf32x3" if args.precision == "tf32x3" else "tc_gemm_tf32"
    rl_heff, _ = roofline(prof, args.steps, clk, tc_kind) if tc_kind in prof else (None, None)
    heff_ms = sum(v["ms"] for k, v in prof.items() if k.startswith("tc_gemm") or k == "zgemm_fp64"
                  or k.startswith("wstage") or k == "prep_operands")
    stages_per_step = st.n_stages / max(args.steps, 1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision if args.precision != "fp64" else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "N": mdl.N, "alpha": mdl.alpha, "h": mdl.h, "m": mdl.m,
                   "chi_max": args.chi, "dt": prm.dt, "segments": prm.seg_len, "precision": args.precision,
                   "krylov": [prm.krylov_max, prm.krylov_tol], "init": "seeded random MPS at chi (seed 0)",
                   "l2": "inputs larger than L2: state + environments %.1f GB" % state_gb(mdl, args.chi),
                   "parallelism": "replicas" if world > 1 else "single GPU, segments batched"},
        "clocks": clk,
        "e2e": {"value": 1.0 / e2e_s, "unit": UNIT, "steps": n_e2e,
                "h2d_bytes_per_step": int(h2d_bytes / n_e2e),
                "d2h_bytes_per_step": int(8 * mdl.N + stages_per_step * (4 + 12 * 8) + 4),
                "what": ("tdvp_init_mps_tensors from pinned host tensors (once per job, its copy amortised "
                         "over the steps) + per step tdvp_step and tdvp_measure(<sigma^z_j>) to host")},
        "gpu_launches": int(st.kernel_launches),
        "roofline": rl,
        "roofline_heff_gemm": rl_heff,
        "heff_tflops": st.heff_flops / max(heff_ms * 1e-3, 1e-12) / 1e12 if heff_ms else None,
        "kernels": {k: {"ms": v["ms"], "launches": v["launches"], "share": v["ms"] / max(ms, 1e-9),
                        "aux": v.get("aux", 0.0)}
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
        "w_total": st.w_total, "chi_max_seen": st.chi_max_seen, "wall_s": wall,
        "autotune": tdvp.autotune_report(),
    }
    if args.fp64_steps > 0 and args.precision != "fp64":
        ref = fp64_reference(args, tdvp, w, mpo, stream)
        ref["speedup"] = value / ref["value"]
        line["fp64_path"] = ref
    if not args.no_cpu_baseline:
        cb = cpu_baseline_sample(args.chi)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "method", "sample")}
        line["cpu_baseline"]["measured_step"] = oracle_step_measured()
    print(json.dumps(line), flush=True)


def fp64_reference(args, tdvp, w, mpo, stream):
    """The plain FP64 GPU path against the mixed path on the same workload and
    from the same seeded state, step by step, for 1 + --fp64-steps steps: every
    step of each path timed with CUDA events on the stream, and after every
    step the largest difference of <sigma^z_j> between the paths (the mixed
    path is held to 1e-5) and both paths' energies (their drift from the
    initial energy is set by the truncation). The FP64 rate excludes the first
    step, which also builds the environments."""
    import torch
    mdl, prm = w.model, w.params
    raw = I.random_mps_tensors(mdl.N, args.chi, seed=0)
    n = args.fp64_steps + 1
    runs = {}
    for prec in (PREC[args.precision], I.FP64):
        mps = tdvp.init_mps_tensors(raw, args.chi, 1e-14)
        p = tdvp.step_params(dt=prm.dt, chi_max=args.chi, w_max=prm.w_max, eps=prm.eps,
                             krylov_max=prm.krylov_max, krylov_tol=prm.krylov_tol, precision=prec,
                             seg_len=prm.seg_len, merge_turning=1)
        e_init = tdvp.energy(mps, mpo)
        ms, sz, en, wt = [], [], [], []
        for _ in range(n):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            st = tdvp.step(mps, mpo, p, 1, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            sz.append(tdvp.measure(mps, tdvp.OBS_SZ))
            en.append(tdvp.energy(mps, mpo))
            wt.append(st.w_total)
        runs[prec] = {"ms": ms, "sz": np.array(sz), "en": np.array(en), "w": np.cumsum(wt), "e_init": e_init}
        del mps
    mx, d = runs[PREC[args.precision]], runs[I.FP64]
    ms_t = d["ms"][1:]
    diff = np.abs(mx["sz"] - d["sz"]).max(axis=1)
    return {
        "value": len(ms_t) / (sum(ms_t) * 1e-3), "unit": UNIT, "steps": len(ms_t), "warmup": 1,
        "ms_per_step": float(np.mean(ms_t)), "dtype": "f64",
        "series": {
            "steps": n,
            "sigma_z_max_abs_diff": [float(v) for v in diff],
            "sigma_z_max_abs_diff_max": float(diff.max()),
            "energy_initial": d["e_init"],
            "energy_drift_mixed": [float(v - mx["e_init"]) for v in mx["en"]],
            "energy_drift_fp64": [float(v - d["e_init"]) for v in d["en"]],
            "energy_abs_diff": [float(v) for v in np.abs(mx["en"] - d["en"])],
            "w_total_mixed": [float(v) for v in mx["w"]],
            "w_total_fp64": [float(v) for v in d["w"]],
            "ms_per_step_mixed": [float(v) for v in mx["ms"]],
        },
    }


def state_gb(mdl, chi):
    dims = [1] + I.bond_dims(mdl.N, chi) + [1]
    site = sum(dims[j] * 2 * dims[j + 1] for j in range(mdl.N)) * 16
    env = sum(2 * dims[j] * dims[j] * mdl.m for j in range(mdl.N)) * 16
    return (site + env) / 1e9


def main():
    args = parse()
    if args.svd_case:
        svd_case(args.svd_case, PREC[args.precision])
        return
    if args.heff_case:
        heff_case(args.heff_case, PREC[args.precision])
        return
    if args.grad_case:
        grad_case(args)
        return
    if args.xxx_case:
        xxx_case(args)
        return
    if args.tdvp1_case:
        tdvp1_case(args)
        return
    if args.tune_case:
        tune_case(args)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
