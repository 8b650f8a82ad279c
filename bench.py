#!/usr/bin/env python3
"""Benchmark of the nonlocal P1 assembly + solve path on GB300.

One step = the whole hot path on one synthetic problem: mesh upload and
precompute, element-pair search and sparsity pattern, quadrature +
deterministic reduction into K, A and b, and the CG solve.  The metric is
element pairs per second of that step (plus p50/p99 step latency), for the
FP32-compensated form, with the plain FP64 form of the same step reported
beside it.  The default workload is the unstructured-like mesh: the Kuhn grid
of the unit cube plus a 3h collar at h = 1/32 with interior vertices jittered
by up to 0.2h (329,232 elements), delta = 3h, fullcaps with 128 Monte Carlo
points.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (under torchrun) runs independent replicas, one per GPU (weak scaling;
the path has no exchange step on one box).  --impl reference times the CPU
oracle (test infrastructure) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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

import nl_inputs as I  # noqa: E402

METRIC = "assembly element-pairs/s; p50/p99 assemble+solve latency, FP32-comp vs FP64"
UNIT = "element-pairs/s"

WORKLOADS = {
    # name: (mesh config, strategy, mc points, seed, CG rtol)
    "cube24_d0125_fullcaps64": ("cube24_d0125", 2, 64, 1, 1e-10),
    "cube6_d025_nocaps": ("cube6_d025", 0, 0, 1, 1e-12),
    "cube16_d016_fullcaps64": ("cube16_d016", 2, 64, 1, 1e-10),
    "jitter38_d3h_fullcaps128": ("jitter38_d3h", 2, 128, 1, 1e-10),
    # the same problem with the quasi-Monte Carlo cap points (not the
    # paper's sampler; see NL_FULLCAPS_QMC)
    "jitter38_d3h_fullcaps_qmc128": ("jitter38_d3h", 6, 128, 1, 1e-10),
    # the same problem under the parabola kernel gamma (1 - |x - y|^2 / delta^2)
    # (a non-constant kernel: every cell and whole element takes the 4-point
    # rule with the kernel at its points)
    "jitter38_d3h_fullcaps128_parabola": ("jitter38_d3h", 2, 128, 1, 1e-10),
}
# kernel shapes phi(s) = c0 + c1 s + c2 s^2 + c3 s^3 of the workloads that have one
WORKLOAD_KERNEL = {"jitter38_d3h_fullcaps128_parabola": (1.0, -1.0, 0.0, 0.0)}
STRAT_NAME = {0: "nocaps", 1: "approxcaps", 2: "fullcaps", 6: "fullcaps_qmc"}

# Algorithmic ALU operations of the quadrature kernels per unit, counted from
# the arithmetic the method prescribes (each 32-bit add, multiply, fused
# multiply-add, compare, min/max, shift or logic operation counts once):
#   per Monte Carlo sample: Philox4x32-10 (10 rounds x (2 mul.lo + 2 mul.hi +
#     4 xor) = 80), the cell choice (6), three uniforms (9), their sort (6),
#     the spacings (4), the point (12) and the ball test (4) = 121;
#   per accepted sample: the barycentrics (16) and the 15 moments (15) = 31;
#   per cut point (1..3 vertices inside): the edge/sphere points, the cells
#     of hull(I u P) with their moments and the cap cell volumes, about 300;
#   per (pair, point): the classification, 4 x 7 = 28.
OPS_PER_SAMPLE = 121
# the quasi-Monte Carlo sampler draws no Philox words: per sample the next
# Sobol' point (4 xor and the lowest set bit, 5) and its shift (4 xor) replace
# the 80 Philox operations
OPS_PER_SAMPLE_QMC = 121 - 80 + 9
OPS_PER_ACCEPTED = 31
OPS_PER_CUT = 300
OPS_PER_PAIR_POINT = 28
ALU_LANES_PER_SM = 128
DEFAULT_WORKLOAD = "jitter38_d3h_fullcaps128"


def entry_errors(K, Kref):
    """Per-entry relative errors of K against Kref (same pattern), with the
    floor of the parity tests for near-zero entries:
    |a - r| / max(|r_ij|, 1e-3 sqrt(|r_ii r_jj|), 1e-7 max_k |r_kk|)."""
    rp, ci, v = K
    rp0, ci0, v0 = Kref
    assert np.array_equal(rp, rp0) and np.array_equal(ci, ci0)
    n = rp.size - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    d = np.zeros(n)
    dm = ci0 == rows
    d[rows[dm]] = np.abs(v0[dm])
    den = np.maximum(np.maximum(np.abs(v0), 1e-3 * np.sqrt(d[rows] * d[ci0])), 1e-7 * d.max())
    return np.abs(v - v0) / np.where(den > 0, den, 1.0)


def _gm_rule_degree5():
    """Grundmann-Moeller rule of degree 5 on the tetrahedron (Grundmann &
    Moeller, SIAM J. Numer. Anal. 15 (1978)): barycentric points, weights
    summing to one."""
    from math import factorial
    s, n = 2, 3
    d = 2 * s + 1
    pts, wts = [], []

    def comps(total, parts):
        if parts == 1:
            yield (total,)
            return
        for i in range(total + 1):
            for rest in comps(total - i, parts - 1):
                yield (i,) + rest
    for i in range(s + 1):
        w = (-1) ** i * 2.0 ** (-2 * s) * (d + n - 2 * i) ** d / (factorial(i) * factorial(d + n - i))
        for beta in comps(s - i, n + 1):
            pts.append([(2 * b + 1) / (d + n - 2 * i) for b in beta])
            wts.append(w * factorial(n))
    return np.array(pts), np.array(wts)


def l2_error(mesh, u_nodal, exact):
    """||u_h - u||_{L2(Omega)}, u_h the P1 interpolant of the nodal solution,
    u = exact(points) (degree-5 Grundmann-Moeller rule per element of Omega)."""
    bary, w = _gm_rule_degree5()
    sel = np.nonzero(mesh.tet_in_omega)[0]
    v = mesh.verts[mesh.tets[sel]]
    e = v[:, 1:] - v[:, :1]
    vol = np.abs(np.einsum("ij,ij->i", e[:, 0], np.cross(e[:, 1], e[:, 2]))) / 6.0
    x = np.einsum("qk,nkd->nqd", bary, v)
    uh = np.einsum("qk,nk->nq", bary, u_nodal[mesh.tets[sel]])
    ue = exact(x)
    return float(np.sqrt(np.sum(vol[:, None] * w[None, :] * (uh - ue) ** 2)))


def l2_error_quadratic(mesh, u_nodal):
    """||u_h - u||_{L2(Omega)} for the manufactured u = |x|^2, u_h the P1
    interpolant of the nodal solution (degree-5 rule per element of Omega)."""
    bary, w = _gm_rule_degree5()
    sel = np.nonzero(mesh.tet_in_omega)[0]
    v = mesh.verts[mesh.tets[sel]]
    e = v[:, 1:] - v[:, :1]
    vol = np.abs(np.einsum("ij,ij->i", e[:, 0], np.cross(e[:, 1], e[:, 2]))) / 6.0
    x = np.einsum("qk,nkd->nqd", bary, v)
    uh = np.einsum("qk,nk->nq", bary, u_nodal[mesh.tets[sel]])
    ue = (x * x).sum(axis=2)
    return float(np.sqrt(np.sum(vol[:, None] * w[None, :] * (uh - ue) ** 2)))


def alu_peak(nl, sm_max_mhz, sms):
    """The k_events roofline's denominator: the measured rate of the
    fullcaps sample's own operation mix (register-only microbenchmark at full
    occupancy, nl_probe_alu_rates), with the per-class rates beside it."""
    rates = nl.probe_alu_rates()
    derived = sms * ALU_LANES_PER_SM * sm_max_mhz * 1e6 / 1e12
    return rates["fullcaps_sample_ops"] / 1e12, {
        "source": "measured: nl_probe_alu_rates, the fullcaps sample's operation mix (a Philox4x32-10 draw, the "
                  "cell choice, three uniforms, their sort, the spacings, the point and the ball test; 121 ops) "
                  "in registers at 64 warps per SM, best of 3",
        "rates_tops": {k: v / 1e12 for k, v in rates.items()},
        "derived_issue_peak_tops": derived,
        "derived_note": "%d SMs x %d lanes x 1 op/clk x %.0f MHz" % (sms, ALU_LANES_PER_SM, sm_max_mhz)}


def _measured_peak(key, fallback):
    """(value, source) from the measured peaks file, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key]), "measured"
    except (OSError, ValueError, KeyError):
        return fallback, "fallback"


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the slowest replica sets the step time)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ws, units_per_rank, t_max_ms):
    """Whole-job throughput of ws independent replicas, each processing
    units_per_rank units, timed by the slowest rank (weak scaling)."""
    return ws * units_per_rank / (t_max_ms / 1e3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _kernel_source_sha():
    h = hashlib.sha256()
    for f in ("nl_quad.cuh", "nl_assemble.cuh", "nl_assemble32.cu"):
        with open(os.path.join(ROOT, "paper_2302_07499_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_record():
    """DRAM bytes per launch of the quadrature kernel from the committed ncu
    summary, or None when the kernel source changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("source_sha") != _kernel_source_sha():
        return None
    return rec.get("dram_bytes_per_step")


def _event_ops(st, qmc=False):
    """ALU operations of the cut-point kernel k_events (cells, caps, samples)."""
    per_sample = OPS_PER_SAMPLE_QMC if qmc else OPS_PER_SAMPLE
    return OPS_PER_CUT * st["cut_points"] + per_sample * st["mc_samples"] + OPS_PER_ACCEPTED * st["mc_accepted"]


def _quadrature_ops(st, qmc=False):
    """ALU operations of the three quadrature kernels."""
    return OPS_PER_PAIR_POINT * 4 * st["pairs"] + _event_ops(st, qmc)


# ---------------------------------------------------------------------------
def run_ours(args, ws, rank, local):
    import torch
    import paper_2302_07499_gb300 as nl

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    cfg, strategy, nmc, seed, rtol = WORKLOADS[args.workload]
    kernel = WORKLOAD_KERNEL.get(args.workload)
    mesh, delta = I.config_mesh(cfg)
    gamma = I.gamma_const(delta)
    g_host = I.quadratic_g(mesh.verts)
    dev = nl.Device()
    d_verts = torch.from_numpy(mesh.verts).cuda()
    d_tets = torch.from_numpy(mesh.tets).cuda()
    d_om = torch.from_numpy(mesh.tet_in_omega).cuda()
    d_free = torch.from_numpy(mesh.node_free).cuda()
    d_g = torch.from_numpy(g_host).cuda()
    d_u = torch.empty(mesh.nv, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(precision, mixed, keep=False):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        m = nl.Mesh(d_verts, d_tets, d_om, d_free, dev)
        ev[1].record(stream)
        p = nl.Pairs(m, delta)
        ev[2].record(stream)
        s = nl.System(p, strategy=strategy, mc_points=nmc, seed=seed, precision=precision, gamma=gamma,
                      f_const=-6.0, g=d_g, kernel=kernel)
        ev[3].record(stream)
        _, info = s.solve(rtol=rtol, mixed=mixed, out=d_u)
        ev[4].record(stream)
        ev[4].synchronize()
        t = [ev[0].elapsed_time(ev[i]) for i in range(1, 5)]
        out = {"total_ms": t[3], "mesh_ms": t[0], "pairs_ms": t[1] - t[0], "assemble_ms": t[2] - t[1],
               "solve_ms": t[3] - t[2], "npairs": p.info["n_pairs"], "stats": s.stats(), "cg": info,
               "nnz_a": p.info["nnz_a"], "n_free": p.info["n_free"], "nnz": p.info["nnz"]}
        if keep:      # outside every timed region: the matrix and the solution for the accuracy report
            out["K"] = s.csr_numpy(nl.MAT_K)
            out["u"] = d_u.cpu().numpy().copy()
        s.close(); p.close(); m.close()
        return out

    def flush_l2():
        flush.zero_()

    # warm-up
    for _ in range(args.warmup):
        flush_l2()
        step(nl.FP32_COMP, True)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = nl.kernel_launches()
    barrier()
    t_wall0 = time.perf_counter()
    steps = []
    for _ in range(args.steps):
        flush_l2()
        steps.append(step(nl.FP32_COMP, True))
    barrier()
    t_wall = time.perf_counter() - t_wall0
    launches = nl.kernel_launches() - launches0
    clocks = sampler.stop()

    ms = [s_["total_ms"] for s_ in steps]
    ms_mean = float(np.mean(ms))
    t_max = max_over_ranks(ms_mean, dist, "cuda")
    npairs = steps[0]["npairs"]
    value = replica_throughput(ws, npairs, t_max)

    # the FP32-comp step once more, untimed, for its matrix and solution
    kept32 = step(nl.FP32_COMP, True, keep=True)

    # FP64 form of the same step (fewer steps: the FP64 pipe is narrow on this
    # part).  Its kernels are warmed up on the small cube6 problem.
    fp64 = None
    accuracy = None
    if args.fp64_steps > 0:
        wm, wd = I.config_mesh("cube6_d025")
        wmesh = nl.Mesh(wm.verts, wm.tets, wm.tet_in_omega, wm.node_free, dev)
        wp = nl.Pairs(wmesh, wd)
        ws_ = nl.System(wp, strategy=strategy, mc_points=nmc, seed=seed, precision=nl.FP64, gamma=I.gamma_const(wd),
                        f_const=-6.0, g=I.quadratic_g(wm.verts))
        ws_.solve(rtol=rtol)
        ws_.close(); wp.close(); wmesh.close()
        r64 = []
        for k in range(args.fp64_steps):
            flush_l2()
            r64.append(step(nl.FP64, False, keep=(k == args.fp64_steps - 1)))
        m64 = float(np.mean([r["total_ms"] for r in r64]))
        fp64 = {"value": npairs / (m64 / 1e3), "unit": UNIT, "ms_per_step": m64,
                "assemble_ms": float(np.mean([r["assemble_ms"] for r in r64])),
                "solve_ms": float(np.mean([r["solve_ms"] for r in r64])),
                "cg_iterations": r64[0]["cg"]["iterations"], "steps": args.fp64_steps,
                "p50_ms": float(np.percentile([r["total_ms"] for r in r64], 50)),
                "p99_ms": float(np.percentile([r["total_ms"] for r in r64], 99))}
        # accuracy of the FP32-comp form against the FP64 form of the same run
        # (the FP64 path matches the CPU oracle to 1e-12 per entry in the
        # parity tests), and of both solutions against the manufactured u
        err = entry_errors(kept32["K"], r64[-1]["K"])
        l2_32 = l2_error_quadratic(mesh, kept32["u"])
        l2_64 = l2_error_quadratic(mesh, r64[-1]["u"])
        accuracy = {"entry_rel_err_fp32comp_vs_fp64": {"max": float(err.max()),
                                                       "p99_9": float(np.percentile(err, 99.9)),
                                                       "entries": int(err.size),
                                                       "bar": 5e-4 if kernel else 1e-5},
                    "l2_error_vs_exact_u": {"fp32comp_mixed_cg": l2_32, "fp64_cg": l2_64,
                                            "ratio": l2_32 / l2_64 if l2_64 > 0 else None, "bar_ratio": 1.01,
                                            "note": "u = |x|^2 solves the constant kernel's problem only; under "
                                                    "the kernel shape only the ratio is meaningful"
                                            if kernel else None},
                    "cg": {"fp32comp_mixed": {"iterations": kept32["cg"]["iterations"],
                                              "refinements": kept32["cg"]["refinements"],
                                              "rel_residual": kept32["cg"]["rel_residual"]},
                           "fp64": {"iterations": r64[-1]["cg"]["iterations"],
                                    "rel_residual": r64[-1]["cg"]["rel_residual"]}},
                    "metric": "per entry |a - r| / max(|r_ij|, 1e-3 sqrt(|r_ii r_jj|), 1e-7 max |r_kk|) over all "
                              "entries of K; L2 over Omega with the degree-5 Grundmann-Moeller rule"}

    # end to end through the C-ABI with host buffers (H2D of the inputs and D2H
    # of the solution inside the timed region)
    e2e_ms = []
    for k in range(max(2, min(args.steps, 5)) + 1):
        flush_l2()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
        p = nl.Pairs(m, delta)
        s = nl.System(p, strategy=strategy, mc_points=nmc, seed=seed, precision=nl.FP32_COMP, gamma=gamma,
                      f_const=-6.0, g=g_host)
        u, _ = s.solve(rtol=rtol, mixed=True)
        t1 = time.perf_counter()
        s.close(); p.close(); m.close()
        if k > 0:
            e2e_ms.append((t1 - t0) * 1e3)
    h2d = mesh.verts.nbytes + mesh.tets.nbytes + mesh.tet_in_omega.nbytes + mesh.node_free.nbytes + g_host.nbytes
    d2h = 8 * mesh.nv
    e2e = {"value": npairs / (float(np.mean(e2e_ms)) / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": float(np.mean(e2e_ms))}

    # SpMV of the CG on this workload's A (HBM-bound when A exceeds L2)
    m = nl.Mesh(d_verts, d_tets, d_om, d_free, dev)
    p = nl.Pairs(m, delta)
    s = nl.System(p, strategy=strategy, mc_points=nmc, seed=seed, precision=nl.FP32_COMP, gamma=gamma,
                  f_const=-6.0, g=d_g)
    hbm = _measured_peak("hbm_gbs", 6800.0)
    spmv = {}
    for name, prec in (("fp64", nl.FP64), ("fp32", nl.FP32_COMP)):
        ms_, by = s.spmv_time(prec, reps=50)
        msc, _ = s.spmv_time(prec, reps=20, flush_bytes=512 * 2 ** 20)
        spmv[name] = {"ms": ms_, "bytes": by, "achieved_gbs": by / (ms_ / 1e3) / 1e9,
                      "frac_of_measured_hbm": by / (ms_ / 1e3) / 1e9 / hbm[0],
                      "cold_l2_ms": msc, "frac_of_measured_hbm_cold_l2": by / (msc / 1e3) / 1e9 / hbm[0]}
    spmv["peak_gbs"] = hbm[0]
    spmv["peak_source"] = hbm[1]
    spmv["a_bytes_fp64"] = int(steps[0]["nnz_a"] * 12)
    spmv["l2_bytes"] = getattr(torch.cuda.get_device_properties(local), "L2_cache_size", None)
    s.close(); p.close(); m.close()

    # roofline of the dominant kernel (the cut-point kernel k_events, which
    # holds the cells, caps and Monte Carlo samples): ALU-bound.  Its duration
    # is the sum over the assembly's chunks of CUDA events recorded on the
    # assembly stream around its launches; the peak is one 32-bit operation
    # per lane per clock on the 128 lanes of every SM at the maximum clock.
    st = steps[-1]["stats"]
    ems = float(np.mean([s_["stats"]["events_ms"] for s_ in steps]))
    qms = float(np.mean([s_["stats"]["quadrature_ms"] for s_ in steps]))
    qmc = strategy == 6
    ops = _event_ops(st, qmc)
    props = torch.cuda.get_device_properties(local)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak, peak_info = alu_peak(nl, sm_max, props.multi_processor_count)
    if qmc:
        # no Philox in the sample: the FP32 fused multiply-add rate bounds the mix
        peak = peak_info["rates_tops"]["ffma_fp32"]
        peak_info = dict(peak_info, source="measured: nl_probe_alu_rates, FP32 fused multiply-add (the "
                         "quasi-Monte Carlo sample draws no Philox words)")
    achieved = ops / (ems / 1e3) / 1e12
    # the FP64 SpMV also needs one FP64 multiply-add per entry: on this part
    # the measured DFMA rate puts a floor under its time next to HBM's
    dfma = peak_info["rates_tops"]["dfma_fp64"] * 1e12
    spmv["fp64"]["dfma_floor_ms"] = steps[0]["nnz_a"] / dfma * 1e3
    spmv["fp64"]["frac_of_measured_dfma"] = spmv["fp64"]["dfma_floor_ms"] / spmv["fp64"]["ms"]
    roofline = {"bound": "alu",
                "kernel": ("k_events<float,%s,kernel shape> + k_whole_shape (the events phase; the operation "
                           "count leaves the rule points of cells and whole elements out)" % STRAT_NAME[strategy])
                if kernel else "k_events<float,%s>" % STRAT_NAME[strategy],
                "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": None if kernel else _traffic_record(),
                "peak_source": peak_info["source"], "peak_detail": peak_info,
                "frac_of_derived_issue_peak": achieved / peak_info["derived_issue_peak_tops"],
                "algorithmic_ops_per_step": ops, "kernel_ms_per_step": ems, "share_of_step": ems / ms_mean,
                "quadrature": {"kernels": "k_classify + k_events + k_combine", "ms": qms,
                               "algorithmic_ops": _quadrature_ops(st, qmc),
                               "achieved_tops": _quadrature_ops(st, qmc) / (qms / 1e3) / 1e12}}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mesh, delta, gamma, strategy, nmc, seed, budget_s=args.cpu_seconds, kernel=kernel)
        one = cpu_baseline(mesh, delta, gamma, strategy, nmc, seed, budget_s=args.cpu_seconds / 2, threads=1,
                           kernel=kernel)
        cpu["one_core"] = {k: one[k] for k in ("value", "unit", "cores", "sample")}

    served = None
    if rank == 0 and ws == 1 and args.serve_requests > 0:
        served = served_comparison(nl, args.serve_requests, args.serve_fp64_requests)

    phases = {k: float(np.mean([s_[k] for s_ in steps])) for k in ("mesh_ms", "pairs_ms", "assemble_ms", "solve_ms")}
    phases["quadrature_ms"] = qms
    for k in ("classify_ms", "events_ms", "combine_ms"):
        phases[k] = float(np.mean([s_["stats"][k] for s_ in steps]))
    phases["reduce_ms"] = float(np.mean([s_["stats"]["reduce_ms"] for s_ in steps]))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload,
                   "mesh": "%s: Kuhn grid%s, %d tets, %d vertices, delta=%g, gamma=15/(2 pi delta^5)"
                   % (cfg, ", interior vertices jittered by up to 0.2h (seed 7)" if cfg.startswith("jitter") else "",
                      mesh.nt, mesh.nv, delta),
                   "strategy": STRAT_NAME[strategy], "mc_points": nmc, "seed": seed,
                   "kernel_shape": ("phi(s) = %g + %g s + %g s^2 + %g s^3, s = min(|x-y|^2/delta^2, 1)" % kernel)
                   if kernel else "constant",
                   "precision": "FP32 per-(pair,point) arithmetic, FP64 accumulation and entries",
                   "solve": "mixed CG (FP32 inner, FP64 residual/updates) to rel. residual %g" % rtol,
                   "element_pairs": npairs, "nnz_K": steps[0]["nnz"], "n_free": steps[0]["n_free"],
                   "nnz_A": steps[0]["nnz_a"], "l2": "flushed before every step (256 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
        "phases_ms": phases,
        "cg": {"iterations": steps[-1]["cg"]["iterations"], "refinements": steps[-1]["cg"]["refinements"],
               "rel_residual": steps[-1]["cg"]["rel_residual"]},
        "fp64": fp64,
        "accuracy": accuracy,
        "roofline": roofline,
        "spmv": spmv,
        "cpu_baseline": cpu,
        "served": served,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "wall_s": t_wall,
        "stats": {k: (int(v) if isinstance(v, int) else v) for k, v in st.items()},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def cpu_baseline(mesh, delta, gamma, strategy, nmc, seed, budget_s=15.0, threads=0, kernel=None):
    """The oracle as it stands, on the host cores (all of them, or `threads`),
    over a bounded contiguous sample of outer elements of the same workload
    (pair search + per-pair blocks + accumulation into K)."""
    import oracle as O
    outer_all = np.nonzero(mesh.tet_in_omega)[0].astype(np.int32)
    cores = threads or O.num_threads()

    def run(outer):
        t0 = time.perf_counter()
        prs = O.pairs(mesh, delta, outer=outer)
        pT, pTp = O.pair_arrays(*prs)
        blocks, _ = O.assemble_blocks(mesh, delta, gamma, strategy, nmc, seed, pT, pTp, nthreads=cores,
                                      kernel=kernel)
        O.blocks_to_matrix(mesh, pT, pTp, blocks)
        return len(pT), time.perf_counter() - t0

    n0 = min(len(outer_all), 64 if cores > 1 else 8)
    np0, t0 = run(outer_all[:n0])
    n1 = int(min(len(outer_all), max(n0, n0 * budget_s / max(t0, 1e-3))))
    npairs, t = run(outer_all[:n1])
    return {"value": npairs / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d of %d outer elements (%d element pairs), %.1f s" % (n1, len(outer_all), npairs, t)}


def run_batch(args, ws, rank, local):
    """Batched assembly of the 256-problem set (1/h ~ U{8..20}, delta/h ~
    U{1,2,3}, strategy ~ U{nocaps, approxcaps, fullcaps-64}, seed 3; FP32-comp
    assembly).  The problems run as consecutive sub-batches of at most
    --batch-pairs element pairs (device memory), each an nl_batch whose launch
    shape is autotuned on the first sub-batch and whose run is a CUDA graph.
    value = all pairs / the summed device time of the batched runs; the same
    problems assembled one by one (nl_assemble) give the solo figure.  The
    first problem of every sub-batch is checked bitwise against its solo
    assembly."""
    import torch
    import paper_2302_07499_gb300 as nl

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    dev = nl.Device()
    small = args.workload == "batch256_small"
    spec = I.batch_problems_small(256, 3) if small else I.batch_problems(256, 3)
    problems = []
    for inv_h, ratio, strat in spec:
        mesh, delta = I.cube_problem(inv_h, ratio)
        kw = dict(strategy=strat, mc_points=64, seed=1, precision=nl.FP32_COMP, gamma=I.gamma_const(delta),
                  f_const=-6.0, g=I.quadratic_g(mesh.verts))
        problems.append((mesh, delta, kw))

    def build(i):
        mesh, delta, _ = problems[i]
        m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
        return m, nl.Pairs(m, delta)

    # solo: each problem alone (pairs built outside the timed call)
    solo_ms, npairs, first_vals = [], [], {}
    for w in range(2):          # one warm-up pass over a few problems, then the timed pass
        rng = range(4) if w == 0 else range(len(problems))
        for i in rng:
            m, p = build(i)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sys_ = nl.System(p, **problems[i][2])
            e1.record(stream)
            e1.synchronize()
            if w == 1:
                solo_ms.append(e0.elapsed_time(e1))
                npairs.append(p.info["n_pairs"])
                first_vals[i] = sys_.csr_numpy(nl.MAT_K)[2].copy()
            sys_.close(); p.close(); m.close()
    # sub-batches of consecutive problems under the pair budget
    groups, cur, acc = [], [], 0
    for i, n_ in enumerate(npairs):
        if cur and acc + n_ > args.batch_pairs:
            groups.append(cur)
            cur, acc = [], 0
        cur.append(i)
        acc += n_
    if cur:
        groups.append(cur)
    batch_ms, shape, checked, equal, launches, tried = [], None, 0, True, 0, None
    l0 = nl.kernel_launches()
    for gi, ids in enumerate(groups):
        built = [build(i) for i in ids]
        b = nl.Batch([(p, problems[i][2]) for i, (m, p) in zip(ids, built)], autotune=(shape is None),
                     use_graph=True, shape=shape)
        info = b.info()
        if shape is None:
            shape = (info["units_per_chunk"], info["classify_threads"])
            tried = info["tried"]
        b.run()                  # warm-up replay
        t = []
        for _ in range(args.steps):
            b.run()
            t.append(b.info()["last_run_ms"])
        batch_ms.append(float(np.mean(t)))
        launches += b.info()["launches_per_run"]
        got = b.system(0).csr_numpy(nl.MAT_K)[2]
        equal &= bool(np.array_equal(got, first_vals[ids[0]]))
        checked += 1
        b.close()
        for m, p in built:
            p.close(); m.close()
    total_pairs = int(sum(npairs))
    value = total_pairs / (sum(batch_ms) / 1e3)
    solo_value = total_pairs / (sum(solo_ms) / 1e3)
    tets = [6 * (inv_h + 2 * r) ** 3 for inv_h, r, _ in spec]
    line = {"metric": "batched assembly element-pairs/s (256 %sproblems)" % ("small " if small else ""),
            "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": 1, "ms_per_step": float(sum(batch_ms)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "problems": len(spec), "tets_min": min(tets),
                       "tets_max": max(tets), "tets_total": int(sum(tets)), "element_pairs": total_pairs,
                       "strategies": {STRAT_NAME[k]: sum(1 for x in spec if x[2] == k) for k in range(3)},
                       "precision": "FP32-comp", "mc_points": 64, "seed": 1,
                       "sub_batches": len(groups), "batch_pairs_budget": args.batch_pairs,
                       "shape": {"units_per_chunk": shape[0], "classify_threads": shape[1]},
                       "autotuner": tried, "graph": True},
            "solo": {"value": solo_value, "ms": float(sum(solo_ms))},
            "speedup_vs_solo": value / solo_value,
            "parity": {"bitwise_equal_to_solo": equal, "problems_checked": checked},
            "gpu_launches": int(launches)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def _serve_stream(nl, reqs, precision, mixed, workers, budget):
    """Replay the arrivals in real time against a fresh server; per request
    (latency, queue delay, service, pairs, status)."""
    srv = nl.Server(budget_bytes=budget, workers=workers, cache=True)
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        dt = r["arrival"] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        req = nl.Server.box_request(r["inv_h"], r["ratio"], strategy=r["strategy"], mc_points=max(1, r["mc"]),
                                    seed=1, precision=precision, mixed=mixed, rtol=1e-10)
        tickets.append(srv.submit(req))
    out = []
    for t in tickets:
        res, _ = srv.wait(t)
        out.append(res)
        srv.release(t)
    srv.close()
    return out


def _serve_summary(res, arrivals_span):
    ok = [r for r in res if r["status"] in (0, 4)]
    lat = np.array([r["t_done"] - r["t_submit"] for r in ok]) * 1e3
    qd = np.array([r["t_start"] - r["t_submit"] for r in ok]) * 1e3
    svc = np.array([r["t_done"] - r["t_start"] for r in ok]) * 1e3
    t_first = min(r["t_submit"] for r in res)
    t_last = max(r["t_done"] for r in res)
    pairs = int(sum(r["n_pairs"] for r in ok))
    makespan = t_last - t_first
    return {"requests": len(res), "completed": len(ok), "failed": len(res) - len(ok),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_queue_ms": float(qd.mean()), "p50_service_ms": float(np.percentile(svc, 50)),
            "element_pairs": pairs, "makespan_s": makespan, "pairs_per_s": pairs / makespan,
            "requests_per_s": len(ok) / makespan, "arrival_span_s": arrivals_span,
            "offered_load": float(svc.sum() / 1e3 / max(arrivals_span, 1e-9)),
            "max_queue_depth": int(max(r["queue_depth_at_start"] for r in ok)),
            "cache_hits": int(sum(r["cache_hit"] for r in ok)),
            "failures": sorted({"%d: %s" % (r["status"], r["message"]) for r in res if r["status"] not in (0, 4)})}


def served_comparison(nl, n_req, n_fp64, workers=4):
    """A prefix of the served request stream (serve_stream_seed5: Poisson
    arrivals at 20/s, mixed sizes, delta/h and strategies), replayed in real
    time in FP32-comp with mixed CG, and its first n_fp64 requests again in
    plain FP64: element pairs/s and p50/p99 latency of the two forms on the
    same requests and the same GPU."""
    reqs = I.request_stream(2000, 20.0, 5)[:n_req]
    budget = 150 * 10 ** 9
    warm = [dict(r, arrival=0.0) for r in sorted(reqs, key=lambda r: r["inv_h"])[:2]]
    _serve_stream(nl, warm, nl.FP32_COMP, True, workers, budget)
    res32 = _serve_stream(nl, reqs, nl.FP32_COMP, True, workers, budget)
    nf = max(2, min(n_fp64, len(reqs)))
    res64 = _serve_stream(nl, reqs[:nf], nl.FP64, False, workers, budget)
    span_f = reqs[nf - 1]["arrival"] - reqs[0]["arrival"]
    s32 = _serve_summary(res32, reqs[-1]["arrival"] - reqs[0]["arrival"])
    s32f = _serve_summary(res32[:nf], span_f)
    s64 = _serve_summary(res64, span_f)
    return {"workload": "serve_stream_seed5: the first %d requests, FP64 on the first %d" % (len(reqs), nf),
            "workers": workers, "fp32_comp": s32, "fp32_comp_same_requests_as_fp64": s32f, "fp64": s64,
            "mixed_over_fp64": {"pairs_per_s": s32f["pairs_per_s"] / s64["pairs_per_s"],
                                "p99_latency": s64["p99_ms"] / s32f["p99_ms"]}}


def run_serve(args, ws, rank, local):
    """The request stream (Poisson arrivals at 20/s, sizes log-uniform in
    10k..400k elements, delta/h ~ U[1,4], 40% fullcaps-128 / 30% approxcaps /
    30% nocaps, seed 5) replayed in real time against the server (150 GB
    budget, --workers concurrent streams): the first --requests requests in
    FP32-comp with mixed CG, and the first --fp64-requests of them again in
    plain FP64 (the same requests).  Latency = completion - submission."""
    import torch
    import paper_2302_07499_gb300 as nl

    torch.cuda.set_device(local)
    reqs = I.request_stream(2000, 20.0, 5)[:args.requests]
    span = reqs[-1]["arrival"] - reqs[0]["arrival"]
    budget = 150 * 10 ** 9
    # warm-up: a few small requests (module load, pools)
    warm = [dict(r, arrival=0.0) for r in sorted(reqs, key=lambda r: r["inv_h"])[:3]]
    _serve_stream(nl, warm, nl.FP32_COMP, True, args.workers, budget)
    sampler = ClockSampler(local)
    sampler.start()
    l0 = nl.kernel_launches()
    res32 = _serve_stream(nl, reqs, nl.FP32_COMP, True, args.workers, budget)
    launches = nl.kernel_launches() - l0
    nf = min(args.fp64_requests, len(reqs))
    res64 = _serve_stream(nl, reqs[:nf], nl.FP64, False, args.workers, budget) if nf > 0 else []
    clocks = sampler.stop()
    s32 = _serve_summary(res32, span)
    s32_prefix = _serve_summary(res32[:nf], reqs[nf - 1]["arrival"] - reqs[0]["arrival"]) if nf > 1 else None
    s64 = _serve_summary(res64, reqs[nf - 1]["arrival"] - reqs[0]["arrival"]) if nf > 1 else None
    line = {"metric": "served assemble+solve: element-pairs/s and p50/p99 latency, FP32-comp vs FP64",
            "value": s32["pairs_per_s"], "unit": UNIT, "n_gpus": ws, "steps": len(reqs), "warmup": len(warm),
            "ms_per_step": s32["makespan_s"] * 1e3 / max(1, s32["completed"]), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serve_stream_seed5", "requests": len(reqs), "rate_per_s": 20.0,
                       "tets": "log-uniform 1e4..4e5", "delta_over_h": "U[1,4]",
                       "strategies": "40% fullcaps-128 / 30% approxcaps / 30% nocaps", "budget_bytes": budget,
                       "workers": args.workers, "cache": True, "solve": "mixed CG to 1e-10 (FP64: plain CG)"},
            "fp32_comp": s32, "fp32_comp_same_prefix_as_fp64": s32_prefix, "fp64": s64,
            "clocks": clocks, "gpu_launches": int(launches)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_spmv(args, ws, rank, local):
    """The CG's SpMV on the jittered 38^3 workload's A (delta = 3h; 29,791
    unknowns, 13.2 M entries): A is assembled (nocaps, FP32-comp: the SpMV
    does not depend on the values' origin), everything but the system is
    released, and the kernel is timed back to back (as in CG, where A partly
    stays in the 129 MB L2) and, launch by launch, after a write of 512 MiB
    that flushes L2 (the HBM-bound figure), after a warm-up of --warmup x 100
    launches.  Small in device memory, so that a profiler can replay it."""
    import torch
    import paper_2302_07499_gb300 as nl

    torch.cuda.set_device(local)
    mesh, delta = I.config_mesh("jitter38_d3h")
    dev = nl.Device()
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    p = nl.Pairs(m, delta)
    s = nl.System(p, strategy=nl.NOCAPS, precision=nl.FP32_COMP, gamma=I.gamma_const(delta), f_const=-6.0)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    hbm = _measured_peak("hbm_gbs", 6800.0)
    out = {}
    for name, prec in (("fp32", nl.FP32_COMP), ("fp64", nl.FP64)):
        # warm-up: a few hundred launches (tens of ms) bring the clocks up;
        # a handful timed straight after a short assembly read 1.5x slower
        s.spmv_time(prec, reps=max(args.warmup, 1) * 100)
        ms_b2b, by = s.spmv_time(prec, reps=max(args.steps, 50))
        ms_cold, _ = s.spmv_time(prec, reps=max(args.steps, 20), flush_bytes=512 * 2 ** 20)
        out[name] = {"bytes": by, "back_to_back_us": ms_b2b * 1e3, "cold_l2_us": ms_cold * 1e3,
                     "frac_of_measured_hbm_back_to_back": by / (ms_b2b / 1e3) / 1e9 / hbm[0],
                     "frac_of_measured_hbm_cold_l2": by / (ms_cold / 1e3) / 1e9 / hbm[0]}
    line = {"metric": "CG SpMV GB/s on the jittered 38^3 workload's A", "unit": "fraction of measured HBM",
            "value": out["fp32"]["frac_of_measured_hbm_back_to_back"], "higher_is_better": True, "n_gpus": ws,
            "config": {"workload": "jitter38_d3h_spmv", "n_free": p.info["n_free"], "nnz_A": p.info["nnz_a"],
                       "kernel": "k_spmv_dot_pad (rows padded to multiples of 4 entries; 16 lanes per row for FP32 values, 8 for FP64; at most the resident blocks)"},
            "hbm_peak_gbs": hbm[0], "hbm_peak_source": hbm[1], "spmv": out}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_fullcaps_variance(args, ws, rank, local):
    """Monte Carlo against quasi-Monte Carlo cap points on the Kuhn 24^3 mesh
    with delta = 1/8 (82,944 tets): for each sampler and cap point count, K
    (FP32-comp) is assembled with 8 seeds, and the spread of its entries over
    the seeds is summarised as the RMS and the maximum over entries of
    std_seeds(K_ij) / sqrt(|K_ii K_jj|), beside the k_events time."""
    import torch
    import paper_2302_07499_gb300 as nl

    torch.cuda.set_device(local)
    mesh, delta = I.config_mesh("cube24_d0125")
    gamma = I.gamma_const(delta)
    dev = nl.Device()
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    p = nl.Pairs(m, delta)
    rows = []
    scale = None
    for name, code in (("fullcaps", nl.FULLCAPS), ("fullcaps_qmc", nl.FULLCAPS_QMC)):
        for nmc in (16, 32, 64, 128):
            vals, ev = [], []
            for seed in range(1, 9):
                s_ = nl.System(p, strategy=code, mc_points=nmc, seed=seed, precision=nl.FP32_COMP, gamma=gamma,
                               f_const=-6.0)
                rp, ci, v = s_.csr(nl.MAT_K)
                vals.append(v.clone())
                ev.append(s_.stats()["events_ms"])
                if scale is None:
                    n = rp.numel() - 1
                    rows_ = torch.repeat_interleave(torch.arange(n, device=v.device), rp[1:] - rp[:-1])
                    dmask = ci.long() == rows_
                    diag = torch.zeros(n, dtype=v.dtype, device=v.device)
                    diag[rows_[dmask]] = v[dmask].abs()
                    # the floor of the entry-error metric: entries of nodes
                    # that no pair reaches (zero diagonal) are not divided by 0
                    scale = torch.clamp(torch.sqrt(diag[rows_] * diag[ci.long()]), min=1e-7 * float(diag.max()))
                s_.close()
            V = torch.stack(vals)
            rel = V.std(dim=0) / scale
            rows.append({"sampler": name, "mc_points": nmc, "events_ms": float(np.mean(ev[1:])),
                         "rms_rel_std": float(torch.sqrt((rel ** 2).mean())),
                         "median_rel_std": float(rel.median()), "p99_rel_std": float(torch.kthvalue(rel.flatten().cpu(), max(1, int(0.99 * rel.numel())))[0]),
                         "max_rel_std": float(rel.max())})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    p.close(); m.close()
    line = {"metric": "spread of K over 8 seeds, Monte Carlo vs quasi-Monte Carlo cap points",
            "unit": "RMS of std/sqrt(|K_ii K_jj|)", "value": None, "n_gpus": ws, "higher_is_better": False,
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": "fullcaps_variance_cube24", "mesh": "cube24_d0125: Kuhn grid, 82944 tets",
                       "delta": delta, "precision": "FP32-comp", "seeds": 8},
            "rows": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)


PAPER3D_STRATEGIES = (("overlap", 4, 0), ("inside", 5, 0), ("barycenter", 3, 0), ("nocaps", 0, 0),
                      ("approxcaps", 1, 0), ("fullcaps", 2, 128))


def run_paper3d(args, ws, rank, local):
    """The shape of the paper's 3D experiment (Sec. 5, Tables 3D_error and
    3D_time): Omega = (0,1)^3, delta = 0.1, kernel integral 3, u = prod
    x_i (1 - x_i) with f = -L u in closed form and g = u on the collar, on
    jittered Kuhn meshes (the stand-in for the unstructured meshes) with
    1/h from --paper3d-inv-h.  Per mesh and strategy: the L2 error of the
    solution (FP32-comp assembly, mixed CG to 1e-10) and the assembly's device
    time (quadrature + reduction); per strategy the efficiency ratio
    lambda_n = -log(e_{n-1}/e_n) / log(t_{n-1}/t_n) between consecutive
    meshes.  On the meshes of --paper3d-unfolded-inv-h the unfolded form of
    Eq. weak0 (every element an outer element, no collar weight) runs beside
    the folded one (rows marked by "form"; lambda uses the folded rows)."""
    import torch
    import paper_2302_07499_gb300 as nl

    torch.cuda.set_device(local)
    dev = nl.Device()
    delta = I.PAPER3D_DELTA
    gamma = I.paper3d_gamma(delta)
    rows = []
    launches0 = nl.kernel_launches()
    unfolded_at = {int(x) for x in args.paper3d_unfolded_inv_h.split(",") if x}
    for inv_h in [int(x) for x in args.paper3d_inv_h.split(",")]:
        mesh = I.paper3d_mesh(inv_h, delta)
        e = mesh.verts[mesh.tets]
        edges = [np.linalg.norm(e[:, a] - e[:, b], axis=1) for a in range(4) for b in range(a + 1, 4)]
        h_avg = float(np.mean(np.concatenate(edges)))
        f = I.paper3d_f(mesh.verts, delta)
        g = I.paper3d_u(mesh.verts)
        forms = ("folded", "unfolded") if inv_h in unfolded_at else ("folded",)
        for form in forms:
            m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev, unfolded=form == "unfolded")
            p = nl.Pairs(m, delta)
            for name, code, nmc in PAPER3D_STRATEGIES:
                sys_ = nl.System(p, strategy=code, mc_points=max(nmc, 1), seed=1, precision=nl.FP32_COMP,
                                 gamma=gamma, f_const=0.0, g=g, f=f)
                st = sys_.stats()
                u, info = sys_.solve(rtol=1e-10, mixed=True)
                rows.append({"inv_h": inv_h, "h_avg": h_avg, "delta_over_h": delta * inv_h, "tets": mesh.nt,
                             "form": form, "element_pairs": p.info["n_pairs"], "strategy": name, "mc_points": nmc,
                             "assembly_ms": st["quadrature_ms"] + st["reduce_ms"],
                             "l2_error": l2_error(mesh, u, I.paper3d_u), "cg_iterations": info["iterations"],
                             "rel_residual": info["rel_residual"]})
                sys_.close()
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            p.close(); m.close()
    lam = {}
    for name, _, _ in PAPER3D_STRATEGIES:
        r = [x for x in rows if x["strategy"] == name and x["form"] == "folded"]
        lam[name] = [-float(np.log(a["l2_error"] / b["l2_error"]) / np.log(a["assembly_ms"] / b["assembly_ms"]))
                     for a, b in zip(r[:-1], r[1:])]
    line = {"metric": "paper 3D experiment shape: L2 error and assembly time per strategy", "unit": "ms, L2 error",
            "value": None, "n_gpus": ws, "higher_is_better": False, "data": "synthetic", "dtype": "f32",
            "config": {"workload": "paper3d_delta01", "omega": "(0,1)^3", "delta": delta,
                       "kernel": "constant, integral 3 over the ball (library gamma = 9/(2 pi delta^3))",
                       "u": "prod x_i (1 - x_i)", "f": "-L u in closed form (nodal, P1-interpolated)",
                       "g": "u at the collar nodes", "mesh": "Kuhn grid of the unit cube plus a ceil(delta/h)-cell "
                       "collar, interior vertices jittered by up to 0.2h (seed 7)",
                       "precision": "FP32-comp assembly, mixed CG to 1e-10"},
            "rows": rows, "lambda": lam, "gpu_launches": int(nl.kernel_launches() - launches0)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle as O
    cfg, strategy, nmc, seed, rtol = WORKLOADS[args.workload]
    kernel = WORKLOAD_KERNEL.get(args.workload)
    mesh, delta = I.config_mesh(cfg)
    gamma = I.gamma_const(delta)
    outer_all = np.nonzero(mesh.tet_in_omega)[0].astype(np.int32)
    cores = O.num_threads()
    # size one step so that warm-up + steps stay within a few minutes
    n_sample = int(os.environ.get("NL_REF_OUTER", "0")) or max(8, min(len(outer_all), 160))

    def one(k):
        sel = outer_all[(k * n_sample) % len(outer_all):][:n_sample]
        t0 = time.perf_counter()
        prs = O.pairs(mesh, delta, outer=sel)
        pT, pTp = O.pair_arrays(*prs)
        blocks, _ = O.assemble_blocks(mesh, delta, gamma, strategy, nmc, seed, pT, pTp, nthreads=cores,
                                      kernel=kernel)
        O.blocks_to_matrix(mesh, pT, pTp, blocks)
        return len(pT), time.perf_counter() - t0

    for k in range(args.warmup):
        one(k)
    res = [one(args.warmup + k) for k in range(args.steps)]
    npairs = sum(r[0] for r in res)
    t = sum(r[1] for r in res)
    value = npairs / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "mesh": cfg, "strategy": STRAT_NAME[strategy], "mc_points": nmc,
                       "seed": seed,
                       "kernel_shape": ("phi(s) = %g + %g s + %g s^2 + %g s^3, s = min(|x-y|^2/delta^2, 1)" % kernel)
                       if kernel else "constant"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d outer elements per step (%d element pairs over %d steps): pair search, "
                                       "per-pair blocks, accumulation into K" % (n_sample, npairs, args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 20, so that the clock sampler sees the timed region; "
                         "5 for batch256_seed3, whose steps take seconds)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + ["batch256_seed3", "serve_stream_seed5",
                                                                           "paper3d_delta01", "batch256_small",
                                                                           "fullcaps_variance_cube24",
                                                                           "jitter38_d3h_spmv"])
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the FP64 form (each takes ~17 s on "
                    "the default workload)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=16,
                    help="default workload: requests of the served-stream comparison after the timed region (0: none)")
    ap.add_argument("--serve-fp64-requests", type=int, default=4,
                    help="default workload: of those, how many are served again in plain FP64")
    ap.add_argument("--requests", type=int, default=300, help="workload serve_stream_seed5: requests replayed")
    ap.add_argument("--fp64-requests", type=int, default=60, help="workload serve_stream_seed5: FP64 prefix")
    ap.add_argument("--workers", type=int, default=4, help="workload serve_stream_seed5: server workers")
    ap.add_argument("--paper3d-inv-h", default="18,21,24,28,32,36,40",
                    help="workload paper3d_delta01: 1/h of the meshes of the sweep")
    ap.add_argument("--paper3d-unfolded-inv-h", default="18,24",
                    help="workload paper3d_delta01: meshes on which the unfolded form runs too")
    ap.add_argument("--batch-pairs", type=float, default=6e8,
                    help="element-pair budget of one sub-batch (workload batch256_seed3)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 5 if args.workload in ("batch256_seed3", "batch256_small") else 20
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload in ("batch256_seed3", "batch256_small"):
        run_batch(args, ws, rank, local)
    elif args.workload == "serve_stream_seed5":
        run_serve(args, ws, rank, local)
    elif args.workload == "paper3d_delta01":
        run_paper3d(args, ws, rank, local)
    elif args.workload == "fullcaps_variance_cube24":
        run_fullcaps_variance(args, ws, rank, local)
    elif args.workload == "jitter38_d3h_spmv":
        run_spmv(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
