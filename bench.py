#!/usr/bin/env python
"""Benchmark of the finite element weak-form evaluator on one GB300.

Workload: linear elasticity ('IK,s(i:j)->I,s(k:l)->K', Tab. ewfd of Cimrman,
arXiv 2107.04121) with vector Q2 hexahedra (27 nodes, 81 x 81 element
matrices) on a 48^3 cube, interior nodes perturbed by +-0.15h (seed 1), 3x3x3
Gauss points, per-element Lame parameters lambda ~ U[0.5, 2], mu ~ U[0.2, 1],
nodal DOFs u ~ N(0, 1).  Synthetic inputs; the paper's own timings use a
1D bar of hexahedra with precomputed geometry on a CPU.

One step = the whole hot path through the C ABI:
  fe_geometry_update (FP64 J, det J, J^-1)  ->  fe_eval_matrix (K_e)
  ->  fe_eval_residual (r_e)  ->  fe_assemble_vector (compensated FP32).
The headline line is the mixed-precision path (FP64 geometry, FP32
contraction); the plain FP64 path is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "elements/s + % roofline, Q2 elasticity K_e & r_e: mixed vs FP64 at rel err ≤1e-5"
UNIT = "elements/s"
Q2_N, Q2_Q = 27, 27
# algorithmic bytes per element of the matrix kernel (FP32 path): read J^-1 and
# w det J (27 qp x 10 floats), the Lame pair (2 doubles), write K_e (81 x 81 floats)
MATRIX_BYTES_PER_ELEM_F32 = Q2_Q * 10 * 4 + 16 + 81 * 81 * 4
MATRIX_BYTES_PER_ELEM_F64 = Q2_Q * 10 * 8 + 16 + 81 * 81 * 8
# the tensor-core matrix kernel that computes the deferred FP64 geometry itself:
# read the 27 x 3 coordinates (gathered, counted once per element), the
# connectivity and the Lame pair; write K_e and the handle's float32 J^-1, w det J
MATRIX_GEO_BYTES_PER_ELEM = Q2_N * 3 * 8 + Q2_N * 4 + 16 + 81 * 81 * 4 + Q2_Q * 10 * 4
# the residual on the stored float32 geometry: read J^-1, w det J, the connectivity,
# the gathered u_e and the Lame pair, write r_e
RESIDUAL_BYTES_PER_ELEM = Q2_Q * 10 * 4 + Q2_N * 4 + 81 * 4 + 16 + 81 * 4


# Navier-Stokes convection 'i,i.j,j' (Eq. fe2) on a 64^3 Q2 cube, +-0.1h seed 3,
# u = a sin(pi x) cos(pi y): residual and the Eq. fe4 derivative K_e(u).
CONVECT_N = 64
# algorithmic bytes per element of the convective matrix kernel: J^-1 and w det J
# (27 points x 10 values), the 27 x 3 gathered velocities, the connectivity,
# and the K_e write (81 x 81)
CV_BYTES_PER_ELEM_F32 = Q2_Q * 10 * 4 + 81 * 4 + 27 * 4 + 81 * 81 * 4
# the FP32 matrix kernel computing the deferred geometry: the 27 nodes' FP64
# coordinates instead of J^-1 and w det J, which it writes as the handle's float32 copy
CV_GEO_BYTES_PER_ELEM_F32 = 27 * 3 * 8 + 81 * 4 + 27 * 4 + 81 * 81 * 4 + Q2_Q * 10 * 4
CV_BYTES_PER_ELEM_F64 = Q2_Q * 10 * 8 + 81 * 8 + 27 * 4 + 81 * 81 * 8
# floating-point operations per element of the sum-factorised convective matrix
# kernel (3x3x3 points, both terms; FMA = 2): interpolation x, y, z stages
# 972 + 1458 + 1944, pointwise 1944, weight contractions z, y 6804 + 20412,
# last contraction and row assembly 56862
CV_FLOPS_PER_ELEM = 972 + 1458 + 1944 + 1944 + 6804 + 20412 + 56862
FP64_PEAK_TFLOPS_NOMINAL = 1.25  # GB300 FP64 (non-tensor), nominal
# DRAM bytes (read + write) of one launch of the step's matrix kernel, per precision
# key "matrix_geo_<prec>", from an ncu capture of the current kernel (the command is
# in profiles/), null for every other size or precision.  The capture runs the
# 32^3 case (32,768 elements: 11.2 MB read + 836.3 MB written in one launch) and is
# scaled to the 110,592 elements of the 48^3 launch by the element count; at 32^3
# up to the 129 MB L2 still holds written lines when the kernel ends, so the
# scaled figure is a lower bound.
MEASURED_TRAFFIC_48 = {"matrix_geo_bf16x3": (11246080 + 836300800) * 110592 // 32768}
# FP64 operations (an FMA counts 2) that the collocation geometry executes for one
# Q2 element with 3x3x3 Gauss points: three 1-D interpolations of 27 lines each
# (6 FMA a line: the middle point is the middle node), J on the points (81 lines of
# a sum, a difference, two multiplies and three FMA in the even-odd form), per point
# 9 cofactors (mul + FMA each) and det J (mul + 2 FMA) -- 1,620 FP64 instructions
GEOMETRY_FLOPS_PER_ELEM_Q2 = 2 * 3 * 27 * 6 + 81 * (4 + 2 * 3) + Q2_Q * (9 * 3 + 5)
GEOMETRY_FP64_INSTR_PER_ELEM_Q2 = 3 * 27 * 6 + 81 * 7 + Q2_Q * (9 * 2 + 3)
# FP64 lanes per clock per SM: a dependent-chain-free DFMA loop measured 1.19 TFLOP/s
# on GB300 at 1.96 GHz over 152 SMs, i.e. 2 lanes per clock per SM
FP64_LANES_PER_CLK_SM = 2


# Adjoint: J = |R|^2 / 2 of the assembled Q2 elasticity residual on a 32^3 cube
# (+-0.1h, seed 4), gradients in lambda_e, mu_e, X and u through torch.autograd.
ADJOINT_N = 32


# Mixed mesh: P1/P2/P3 tetrahedra (200k/120k/40k, Delaunay, GM rules of index p)
# and Q1/Q2/Q3 hexahedra (60k/30k/8k, +-0.1h), weighted Laplace, weighted mass
# and Lame elasticity matrices of every group in one persistent launch.
MIXED_FORMS = ("laplace", "mass", "elasticity")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=48, help="cube edge in elements (48 -> 110,592 hexes)")
    ap.add_argument("--workload", choices=["elasticity", "convection", "mixed", "paths", "fp64units"],
                    default="elasticity",
                    help="convection: only the Navier-Stokes convection workload on an n^3 cube (both "
                         "precisions); mixed: only the mixed-mesh batch; paths: each mixed-mesh item's matrix "
                         "on the CUDA-core and the tensor-core contraction path, timed apart; fp64units: the "
                         "DFMA and FP64 MMA rates (fe_diag_fp64); no oracle, one JSON line")
    ap.add_argument("--scale", type=float, default=1.0, help="mixed and paths workloads: scale of every group")
    ap.add_argument("--groups", default="", help="paths workload: comma-separated groups (e.g. Q2,Q3); all if empty")
    ap.add_argument("--prec", default="auto",
                    help="contraction precision of the headline path; auto = fastest of the ladder within 1e-5")
    ap.add_argument("--skip-extras", action="store_true",
                    help="time the headline path only (no FP64 path, e2e, CPU baseline, error check)")
    return ap.parse_args()


# ---- distributed plumbing (replicas: every rank evaluates its own mesh) -------------

def dist_setup(args, backend=None):
    """One process per GPU from torchrun's environment: NCCL on GPUs (gloo where there
    is none, e.g. the multi-process tests on the host)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = backend or ("nccl" if torch.cuda.is_available() else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    """The maximum of x over the ranks (the job's time is its slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(step_ms, units_per_step, steps, ws):
    """Whole-job throughput of replicas: every rank processes units_per_step per step,
    the job takes as long as its slowest rank (max over ranks of the summed step times).
    Returns (units per second, ms per step)."""
    total_ms = max_over_ranks(sum(step_ms), ws)
    return ws * units_per_step * steps / (total_ms / 1e3), total_ms / steps


# ---- clocks --------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        # under load: samples drawing more than the median power
        pw = sorted(r[2] for r in rows)
        thr = pw[len(pw) // 2]
        load = [r for r in rows if r[2] >= thr] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "reasons": reasons, "samples": len(rows)}


# ---- workload --------------------------------------------------------------------------

class Workload:
    def __init__(self, n, device):
        import torch

        from paper_2107_04121_gb300 import fe, meshgen
        self.fe, self.torch = fe, torch
        self.mesh, self.lam, self.mu, self.u = meshgen.elasticity_q2_cube(n, seed=1)
        self.E = self.mesh.n_elems
        self.ctx = fe.Context(device)
        self.coords = torch.from_numpy(self.mesh.coords).to(device)
        self.conn = torch.from_numpy(self.mesh.conn).to(device)
        self.m = fe.Mesh(self.coords, self.conn)
        # each path keeps only the geometry copy it reads; the mixed step uses a
        # deferred float32-only handle, whose geometry the residual kernel computes
        self.geoms = {"f64": fe.hex_geometry(self.ctx, self.m, 2, 3, flags=fe.GEOM_STORE_F64),
                      "f32": fe.hex_geometry(self.ctx, self.m, 2, 3, flags=fe.GEOM_STORE_F32),
                      "f32d": fe.hex_geometry(self.ctx, self.m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)}
        self.form = fe.elasticity_form(fe.MAT_LAME)
        self.mat = torch.from_numpy(np.stack([self.lam, self.mu], 1)).to(device)
        self.u64 = torch.from_numpy(self.u).to(device)
        self.u32 = self.u64.float()
        self.asm = fe.assembly_create(self.ctx, self.m)
        self.bufs = {}
        self.ctx.check()

    def outputs(self, prec):
        torch = self.torch
        f64 = prec == "f64"
        if prec not in self.bufs:
            dt = torch.float64 if f64 else torch.float32
            self.bufs[prec] = (torch.empty((self.E, 81, 81), dtype=dt, device="cuda"),
                               torch.empty((self.E, 81), dtype=dt, device="cuda"),
                               torch.zeros(self.mesh.n_nodes * 3, dtype=dt, device="cuda"))
        return self.bufs[prec]

    def drop(self, prec):
        self.bufs.pop(prec, None)
        self.torch.cuda.empty_cache()

    @staticmethod
    def matrix_first(prec):
        """Tensor-core precisions: the matrix kernel computes the stale deferred FP64
        geometry itself (beside the K_e stream) and the residual reads its float32
        copy; otherwise the residual kernel computes it and the matrix follows."""
        return prec in ("tf32x3", "bf16x3", "bf16")

    def parts(self, prec):
        if self.matrix_first(prec):
            return ("matrix_with_geometry", "residual", "assembly")
        return ("geometry_and_residual", "matrix", "assembly")

    def step(self, prec, ev=None):
        """One step; `ev` (optional) gets four CUDA events recorded at the start and
        after each of the three parts (parts(prec) names them)."""
        fe = self.fe
        K, r, g = self.outputs(prec)
        rec = (lambda i: ev[i].record()) if ev else (lambda i: None)
        rec(0)
        geom = self.geoms["f64" if prec == "f64" else "f32d"]
        u = self.u64 if prec == "f64" else self.u32
        geom.update()
        if self.matrix_first(prec):
            fe.eval_matrix(self.ctx, self.form, geom, [self.mat, None, None], prec, out=K)
            rec(1)
            fe.eval_residual(self.ctx, self.form, geom, [self.mat, None, u], prec, out=r)
        else:
            # FP64: the geometry kernel (an eager handle); f32: the stale deferred
            # geometry computed by the residual kernel, whose copy the matrix reads
            fe.eval_residual(self.ctx, self.form, geom, [self.mat, None, u], prec, out=r)
            rec(1)
            fe.eval_matrix(self.ctx, self.form, geom, [self.mat, None, None], prec, out=K)
        rec(2)
        fe.assemble_vector(self.ctx, self.asm, 3, r, prec, out=g,
                           flags=0 if prec == "f64" else fe.ASSEMBLE_COMPENSATED)
        rec(3)


def kernels_per_step(prec):
    # FP64: geometry, residual, matrix, assembly; tensor-core precisions: the matrix
    # kernel computing the geometry, the residual, the assembly; f32: geometry +
    # residual in one kernel, matrix, assembly
    return 4 if prec == "f64" else 3
LADDER = ["f32", "tf32x3", "bf16x3", "bf16"]
DEFAULT_MIXED = "bf16x3"


def precision_ladder(wl, flush, reps=5):
    """Matrix-kernel time of each contraction precision of the mixed path (FP64
    geometry in every case).  Each rung then runs one whole step whose outputs stay
    resident for the error check over every element."""
    torch = wl.torch
    out = {}
    for p in LADDER:
        K, r, g = wl.outputs(p)
        geom = wl.geoms["f32"]
        for _ in range(2):
            wl.fe.eval_matrix(wl.ctx, wl.form, geom, [wl.mat, None, None], p, out=K)
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            wl.fe.eval_matrix(wl.ctx, wl.form, geom, [wl.mat, None, None], p, out=K)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        wl.step(p)
        out[p] = {"matrix_ms": statistics.median(ts)}
    wl.ctx.check()
    return out


def every_element_errors(wl, precs, chunk=13824):
    """Part of the CPU-baseline leg (rank 0, N = 1, outside every timed region):
    the FP64 oracle computes K_e and r_e of all elements on the host cores, chunk
    by chunk, and each precision's resident step outputs are compared with them:
    max over elements of ||K_e - K_ref||_F / ||K_ref||_F, and ||r - r_ref||_2 /
    ||r_ref||_2 over the array.  The differences are formed in float64 on the
    device (the oracle's values are uploaded; nothing flows the other way)."""
    import oracle
    torch = wl.torch
    ref = oracle.RefElement(2, 3)
    worst = {p: 0.0 for p in precs}
    rnum = {p: 0.0 for p in precs}
    rden = 0.0
    for c0 in range(0, wl.E, chunk):
        c1 = min(wl.E, c0 + chunk)
        conn = np.ascontiguousarray(wl.mesh.conn[c0:c1])
        wdetJ, G, _ = oracle.geometry(wl.mesh.coords, conn, ref)
        D = oracle.lame_to_D(wl.lam[c0:c1], wl.mu[c0:c1])
        Kref = torch.from_numpy(oracle.matrix_elasticity(wdetJ, G, D)).cuda()
        rref = torch.from_numpy(oracle.residual_elasticity(conn, wdetJ, G, D, wl.u)).cuda()
        del wdetJ, G
        kden = (Kref * Kref).sum((1, 2))
        rden += float((rref * rref).sum())
        for p in precs:
            K, r, _ = wl.bufs[p]
            d = K[c0:c1].double() - Kref
            worst[p] = max(worst[p], float(((d * d).sum((1, 2)) / kden).sqrt().max()))
            del d
            dr = r[c0:c1].double() - rref
            rnum[p] += float((dr * dr).sum())
        del Kref, rref, kden
    torch.cuda.empty_cache()
    out = {}
    for p in precs:
        out["K_" + p] = worst[p]
        out["r_" + p] = float(np.sqrt(rnum[p] / rden))
    return out


def timed_steps(wl, prec, steps, warmup, ws, flush):
    """Per-step CUDA-event times (ms), matrix-kernel times (ms) and the mean
    time of each part of the step; L2 flushed between steps."""
    torch = wl.torch
    for _ in range(warmup):
        wl.step(prec)
    wl.ctx.check()
    barrier(ws)
    torch.cuda.synchronize()
    ev = []
    for _ in range(steps):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        wl.step(prec, e)
        ev.append(e)
    torch.cuda.synchronize()
    barrier(ws)
    wl.ctx.check()
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    mi = 0 if wl.matrix_first(prec) else 1
    mat_ms = [e[mi].elapsed_time(e[mi + 1]) for e in ev]
    parts = {name: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in ev)
             for i, name in enumerate(wl.parts(prec))}
    return step_ms, mat_ms, parts


def time_call(wl, flush, fn, reps=5, warmup=2):
    """Median CUDA-event time (ms) of fn, L2 flushed before each call."""
    torch = wl.torch
    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    wl.ctx.check()
    return statistics.median(ts)


def rel_matrix_error(K, Kref):
    """max over elements of ||K_e - K_e^ref||_F / ||K_e^ref||_F."""
    K = np.asarray(K, dtype=np.float64)
    num = np.sqrt(((K - Kref) ** 2).sum((1, 2)))
    den = np.sqrt((Kref ** 2).sum((1, 2)))
    return float((num / den).max()) if len(den) else 0.0


def rel_vector_error(r, rref):
    """||r - r_ref||_2 / ||r_ref||_2 over the whole array."""
    r = np.asarray(r, dtype=np.float64).ravel()
    rref = np.asarray(rref).ravel()
    return float(np.linalg.norm(r - rref) / np.linalg.norm(rref))


def sampled_errors(wl, precs, ref):
    """Relative errors of the GPU outputs on the sampled elements of `ref`
    (computed by the oracle in the CPU-baseline leg)."""
    if ref is None:
        return {}, 0
    idx, Kref, rref = ref
    out = {}
    it = wl.torch.from_numpy(idx).cuda()
    for p in precs:
        K, r, _ = wl.outputs(p)
        out["K_" + p] = rel_matrix_error(K[it].double().cpu().numpy(), Kref)
        out["r_" + p] = rel_vector_error(r[it].double().cpu().numpy(), rref)
    return out, len(idx)


def e2e_job_summary(per_ms, units, h2d, d2h, ws):
    """The job's end-to-end figures from one rank's step times: the link is shared with
    the host, so a rank's step is its median (mean and worst beside it); the job's step
    is the slowest rank's, and the rate and the bytes moved are the whole job's."""
    ms = max_over_ranks(statistics.median(per_ms), ws)
    return {"value": ws * units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "mean_ms": max_over_ranks(statistics.mean(per_ms), ws), "max_ms": max_over_ranks(max(per_ms), ws),
            "h2d_bytes_per_step": ws * h2d, "d2h_bytes_per_step": ws * d2h}


def e2e_measure(wl, prec, steps, ws=1, chunks=8):
    """Same step through the public API with host buffers: pinned H2D of the inputs
    (coordinates, connectivity, materials, DOFs) and D2H of every result (K_e, r_e,
    assembled vector), all inside the CUDA-event timed region.  The mesh is
    evaluated in `chunks` element ranges (geometry views) so that the transfer of
    one range's K_e, on a second stream, overlaps the evaluation of the next: the
    step is bound by the device-to-host link.  Every rank measures its replica; the
    job's step is the slowest rank's, and the rate and the bytes are the job's."""
    torch, fe = wl.torch, wl.fe
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_in = [pin(wl.mesh.coords), pin(wl.mesh.conn), pin(np.stack([wl.lam, wl.mu], 1)),
            pin(wl.u.astype(np.float32) if prec != "f64" else wl.u)]
    u_dev = wl.u32 if prec != "f64" else wl.u64
    d_in = [wl.coords, wl.conn, wl.mat, u_dev]
    K, r, g = wl.outputs(prec)
    h_out = [torch.empty(K.shape, dtype=K.dtype).pin_memory(), torch.empty(r.shape, dtype=r.dtype).pin_memory(),
             torch.empty(g.shape, dtype=g.dtype).pin_memory()]
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    d2h = sum(t.numel() * t.element_size() for t in h_out)
    geom = wl.geoms["f64" if prec == "f64" else "f32"]
    E = wl.E
    EC = (E + chunks - 1) // chunks
    ranges = [(e0, min(E, e0 + EC)) for e0 in range(0, E, EC)]
    views = [geom.view(e0, e1 - e0) for e0, e1 in ranges]
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream()

    def one():
        for d, h in zip(d_in, h_in):
            d.copy_(h, non_blocking=True)
        for (e0, e1), v in zip(ranges, views):
            v.update()  # FP64 geometry of this element range
            fe.eval_matrix(wl.ctx, wl.form, v, [wl.mat[e0:e1], None, None], prec, out=K[e0:e1])
            ev = torch.cuda.Event()
            ev.record(comp)
            copy.wait_event(ev)
            with torch.cuda.stream(copy):
                h_out[0][e0:e1].copy_(K[e0:e1], non_blocking=True)
        fe.eval_residual(wl.ctx, wl.form, geom, [wl.mat, None, u_dev], prec, out=r)
        fe.assemble_vector(wl.ctx, wl.asm, 3, r, prec, out=g, flags=0 if prec == "f64" else fe.ASSEMBLE_COMPENSATED)
        ev = torch.cuda.Event()
        ev.record(comp)
        copy.wait_event(ev)
        with torch.cuda.stream(copy):
            h_out[1].copy_(r, non_blocking=True)
            h_out[2].copy_(g, non_blocking=True)
        comp.wait_stream(copy)

    for _ in range(2):  # warm-up: first touches of the pinned buffers, the views
        one()
    torch.cuda.synchronize()
    barrier(ws)
    per = []
    for _ in range(steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        one()
        b.record()
        b.synchronize()
        per.append(a.elapsed_time(b))
    wl.ctx.check()
    for v in views:
        v.free()
    return {**e2e_job_summary(per, wl.E, h2d, d2h, ws), "chunks": len(ranges),
            "note": "bound by the device-to-host link (about 194 GB/s for pinned copies and for SM stores to "
                    "host memory on this machine)"}


class ConvectWorkload:
    """Navier-Stokes convection, one step = FP64 geometry -> K_e(u) (Eq. fe4) ->
    r_e(u) (Eq. fe2) -> assembled residual (compensated FP32 / FP64)."""

    def __init__(self, n, device):
        import torch

        from paper_2107_04121_gb300 import fe, meshgen
        self.fe, self.torch = fe, torch
        self.mesh, self.u = meshgen.convect_q2_cube(n, seed=3)
        self.E = self.mesh.n_elems
        self.ctx = fe.Context(device)
        self.coords = torch.from_numpy(self.mesh.coords).to(device)
        self.conn = torch.from_numpy(self.mesh.conn).to(device)
        self.m = fe.Mesh(self.coords, self.conn)
        self.geoms = {"f64": fe.hex_geometry(self.ctx, self.m, 2, 3, flags=fe.GEOM_STORE_F64),
                      "f32": fe.hex_geometry(self.ctx, self.m, 2, 3, flags=fe.GEOM_STORE_F32 | fe.GEOM_DEFERRED)}
        self.form = fe.convect_form()
        self.u64 = torch.from_numpy(self.u).to(device)
        self.u32 = self.u64.float()
        self.asm = fe.assembly_create(self.ctx, self.m)
        self.bufs = {}
        self.ctx.check()

    outputs = Workload.outputs
    drop = Workload.drop

    @staticmethod
    def matrix_first(prec):
        """FP32: the matrix kernel computes the stale deferred FP64 geometry (its FP64
        stages beside the other CTAs' float32 contractions) and the residual reads the
        float32 copy."""
        return prec == "f32"

    def parts(self, prec):
        if self.matrix_first(prec):
            return ("geometry_and_matrix", "residual", "assembly")
        return ("geometry_and_residual", "matrix", "assembly")

    def step(self, prec, ev=None):
        """FP32: the deferred geometry is computed (FP64) by the matrix kernel, then
        r_e(u) and the assembly; FP64: geometry kernel, residual, K_e(u), assembly."""
        fe = self.fe
        K, r, g = self.outputs(prec)
        u = self.u64 if prec == "f64" else self.u32
        rec = (lambda i: ev[i].record()) if ev else (lambda i: None)
        geom = self.geoms[prec]
        rec(0)
        geom.update()
        if self.matrix_first(prec):
            fe.eval_matrix(self.ctx, self.form, geom, [None, u, u], prec, out=K)
            rec(1)
            fe.eval_residual(self.ctx, self.form, geom, [None, u, u], prec, out=r)
        else:
            fe.eval_residual(self.ctx, self.form, geom, [None, u, u], prec, out=r)
            rec(1)
            fe.eval_matrix(self.ctx, self.form, geom, [None, u, u], prec, out=K)
        rec(2)
        fe.assemble_vector(self.ctx, self.asm, 3, r, prec, out=g,
                           flags=0 if prec == "f64" else fe.ASSEMBLE_COMPENSATED)
        rec(3)


def convect_measure(n, device, ws, flush, ref, hbm_peak, steps=5, warmup=3):
    """FP32 and FP64 steps of the convection workload, the roofline of its matrix
    kernel (HBM for FP32, the FP64 pipe for FP64) and sampled errors against the
    oracle (reference computed in the CPU-baseline leg)."""
    cw = ConvectWorkload(n, device)
    out = {"workload": "Navier-Stokes convection 'i,i.j,j', Q2 hexahedra, %d^3 = %d elements, +-0.1h seed 3, "
                       "u = a sin(pi x) cos(pi y); step = FP64 geometry (FP32: computed by the matrix "
                       "kernel) + K_e(u) (Eq. fe4) + r_e(u) + assembly" % (n, cw.E), "elements": cw.E}
    for prec in ("f32", "f64"):
        st, mt, parts = timed_steps(cw, prec, steps, warmup, ws, flush)
        t = max_over_ranks(sum(st), ws)
        mat = sum(mt) / len(mt)
        d = {"value": ws * cw.E * steps / (t / 1e3), "unit": UNIT, "ms_per_step": t / steps, "matrix_ms": mat,
             "parts_ms": parts}
        if prec == "f32":
            b_el = CV_GEO_BYTES_PER_ELEM_F32 if cw.matrix_first(prec) else CV_BYTES_PER_ELEM_F32
            ach = cw.E * b_el / (mat / 1e3) / 1e9
            d["roofline"] = {"kernel": "k_convect_sf (matrix, f32%s)" % (", computing the deferred FP64 geometry"
                                                                        if cw.matrix_first(prec) else ""),
                             "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                             "frac": ach / hbm_peak, "bytes_per_elem": b_el}
            if cw.matrix_first(prec):
                # the same matrix kernel on the stored float32 geometry (the handle is
                # current after the steps), timed alone
                K, _, _ = cw.outputs(prec)
                geom = cw.geoms[prec]
                t_m = time_call(cw, flush, lambda: cw.fe.eval_matrix(cw.ctx, cw.form, geom, [None, cw.u32, cw.u32],
                                                                     prec, out=K))
                a2 = cw.E * CV_BYTES_PER_ELEM_F32 / (t_m / 1e3) / 1e9
                d["matrix_stored_geometry"] = {"ms": t_m, "roofline": {
                    "kernel": "k_convect_sf (matrix, f32, stored geometry)", "bound": "hbm", "achieved": a2,
                    "peak": hbm_peak, "unit": "GB/s", "frac": a2 / hbm_peak, "bytes_per_elem": CV_BYTES_PER_ELEM_F32}}
        else:
            ach = cw.E * CV_FLOPS_PER_ELEM / (mat / 1e3) / 1e12
            d["roofline"] = {"kernel": "k_convect_sf (matrix, f64)", "bound": "fp64", "achieved": ach,
                             "peak": FP64_PEAK_TFLOPS_NOMINAL, "peak_source": "nominal", "unit": "TFLOP/s",
                             "frac": ach / FP64_PEAK_TFLOPS_NOMINAL, "flops_per_elem": CV_FLOPS_PER_ELEM}
        if ref is not None:
            errs, ns = sampled_errors(cw, [prec], ref)
            d["rel_err_K"], d["rel_err_r"], d["sampled_elements"] = errs["K_" + prec], errs["r_" + prec], ns
        out[prec] = d
        cw.drop(prec)
    cw.ctx.check()
    cw.ctx.close()
    return out


def adjoint_measure(n, device, flush, ref, steps=5, warmup=3):
    """One gradient step = forward (FP64 geometry, r_e, assembly, J) + backward
    (geometry recomputed, K Rbar for du, adjoint kernel, assembly of dX), in FP32
    (the geometry computed by the residual kernels) and FP64, with the adjoint
    kernel timed alone; errors against the oracle gradient (computed in the
    CPU-baseline leg)."""
    import torch

    from paper_2107_04121_gb300 import autograd as fad
    from paper_2107_04121_gb300 import fe, meshgen
    mesh, lam, mu, u = meshgen.elasticity_q2_cube(n, seed=4, perturb=0.1)
    ctx = fe.Context(device)
    out = {"workload": "J = |R|^2/2 of the assembled Q2 elasticity residual, %d^3 = %d hexes, +-0.1h seed 4; "
                       "step = forward + backward (d/dlambda, d/dmu, d/dX, d/du)" % (n, mesh.n_elems),
           "elements": mesh.n_elems}
    for prec in ("f32", "f64"):
        X = torch.from_numpy(mesh.coords).to(device)
        conn = torch.from_numpy(mesh.conn).to(device)
        prob = fad.ElasticityProblem(ctx, X, conn, 2, 3, prec)
        dt = prob.dtype
        lam_t = torch.from_numpy(lam).to(device, dt).requires_grad_()
        mu_t = torch.from_numpy(mu).to(device, dt).requires_grad_()
        u_t = torch.from_numpy(u).to(device, dt).requires_grad_()
        X.requires_grad_()

        def one():
            for t in (lam_t, mu_t, X, u_t):
                t.grad = None
            R = fad.assembled_elasticity_residual(prob, lam_t, mu_t, X, u_t)
            Jv = 0.5 * (R.double() * R.double()).sum()
            Jv.backward()
            return Jv

        for _ in range(warmup):
            one()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            one()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        # the adjoint kernel alone
        mat = torch.stack([lam_t.detach(), mu_t.detach()], 1).double().contiguous()
        rbar = torch.randn(3 * mesh.n_nodes, dtype=dt, device=device)
        kt = []
        for i in range(warmup + steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fe.eval_residual_adjoint(ctx, prob.form, prob.geom, [mat, None, u_t.detach()], rbar, prec)
            b.record()
            b.synchronize()
            if i >= warmup:
                kt.append(a.elapsed_time(b))
        ctx.check()
        ms = statistics.median(ts)
        d = {"value": mesh.n_elems / (ms / 1e3), "unit": UNIT + " (gradient steps x elements)", "ms_per_step": ms,
             "adjoint_kernel_ms": statistics.median(kt)}
        if ref is not None:
            one()
            Jref, dl, dm, dX = ref
            rel = lambda a, b: float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / np.linalg.norm(b))
            d["rel_err"] = {"lambda": rel(lam_t.grad.cpu().numpy(), dl), "mu": rel(mu_t.grad.cpu().numpy(), dm),
                            "X": rel(X.grad.cpu().numpy(), dX)}
        out[prec] = d
        del prob
    ctx.close()
    return out


def mixed_setup(scale, device):
    import torch

    from paper_2107_04121_gb300 import fe, meshgen
    ctx = fe.Context(device)
    groups = []
    for name, mesh in meshgen.mixed_mesh_groups(scale, seed=2):
        p = int(name[1])
        coords = torch.from_numpy(mesh.coords).to(device)
        m = fe.Mesh(coords, torch.from_numpy(mesh.conn).to(device))
        geom = (fe.tet_geometry(ctx, m, p, flags=fe.GEOM_STORE_F32) if name[0] == "P" else
                fe.hex_geometry(ctx, m, p, p + 1, flags=fe.GEOM_STORE_F32))
        rng = np.random.default_rng(100 + p + (10 if name[0] == "P" else 0))
        coef = rng.uniform(0.5, 2.0, mesh.n_elems)
        lam, mu = rng.uniform(0.5, 2.0, mesh.n_elems), rng.uniform(0.2, 1.0, mesh.n_elems)
        groups.append({"name": name, "mesh": mesh, "m": m, "geom": geom, "coef": coef, "lam": lam, "mu": mu,
                       "mats": {"laplace": torch.from_numpy(coef).to(device),
                                "mass": torch.from_numpy(coef).to(device),
                                "elasticity": torch.from_numpy(np.stack([lam, mu], 1)).to(device)}})
    forms = {"laplace": fe.laplace_form(weighted=True), "mass": fe.mass_form(1, weighted=True),
             "elasticity": fe.elasticity_form(fe.MAT_LAME)}
    return ctx, groups, forms


def mixed_measure(device, flush, ref, steps=5, warmup=3, scale=1.0):
    """The mixed-mesh batch: one CUDA-graph launch = FP64 geometry of the six
    groups + the matrices of all 18 (group, form) items under the autotuned
    schedule (persistent class kernels or one launch per item); beside it each
    schedule's matrix launches alone, the same work as separate per-item calls
    from Python, and the chosen schedule's matrices against the HBM roofline."""
    import torch

    from paper_2107_04121_gb300 import fe
    ctx, groups, forms = mixed_setup(scale, device)
    items = [(g["geom"], forms[f], g["mats"][f], None) for g in groups for f in MIXED_FORMS]
    t0 = time.perf_counter()
    batch = fe.Batch(ctx, items, fe.BATCH_AUTOTUNE | fe.BATCH_GRAPH | fe.BATCH_GEOMETRY)
    plan_s = time.perf_counter() - t0
    same_out = [(g, f, m, K) for (g, f, m, _), K in zip(items, batch.outputs)]
    mats_p = fe.Batch(ctx, same_out, fe.BATCH_AUTOTUNE | fe.BATCH_PERSISTENT)
    mats_l = fe.Batch(ctx, same_out, fe.BATCH_AUTOTUNE | fe.BATCH_LAUNCHES)  # contraction paths tuned

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    def separate():
        for g in groups:
            g["geom"].update()
        for (g, f, m, _), K in zip(items, batch.outputs):
            fe.eval_matrix(ctx, f, g, [m, None, None], "f32", out=K)

    ms_graph = timed(batch.run)
    ms_persistent = timed(mats_p.run)
    ms_launches = timed(mats_l.run)
    ms_sep = timed(separate)
    schedule = batch.schedule()
    ms_kernel = ms_launches if schedule == "launches" else ms_persistent
    ctx.check()
    n_el = sum(g["mesh"].n_elems for g in groups)
    # algorithmic bytes of the matrices: J^-1 and w det J of each group once (FP32,
    # Q x 10 values per element; the job needs them once however many forms read
    # them), and per item and element the material (8 or 16 B) and the K_e write
    kbytes = 0
    seen = set()
    for (g, f, m, _), K in zip(items, batch.outputs):
        E = K.shape[0]
        if id(g) not in seen:
            seen.add(id(g))
            kbytes += E * g.Q * 10 * 4
        kbytes += E * (m.element_size() * m.numel() // max(E, 1) + K[0].numel() * 4)
    paths = [batch.describe(k)["path"] for k in range(len(items))]
    launches = len(items) - sum("shared" in p for p in paths) // 2
    out = {"workload": "mixed mesh: P1/P2/P3 tets %s, Q1/Q2/Q3 hexes %s; weighted Laplace + weighted mass + Lame "
                       "elasticity matrices, FP32 from FP64 geometry" % (
                           "/".join(str(g["mesh"].n_elems) for g in groups[:3]),
                           "/".join(str(g["mesh"].n_elems) for g in groups[3:])),
           "elements": n_el, "items": len(items), "plan_seconds": plan_s,
           "graph_ms": ms_graph, "value": n_el / (ms_graph / 1e3), "unit": UNIT + " (all 3 forms per element)",
           "schedule": schedule, "persistent_kernels_ms": ms_persistent, "per_item_launches_ms": ms_launches,
           "separate_calls_ms": ms_sep,
           "roofline": {"kernel": ("the items' matrix kernels on 3 streams, %d launches (elasticity and Laplacian "
                                   "items of a geometry sharing one launch where the autotuner paired them)"
                                   % launches if schedule == "launches"
                                   else "k_batch, persistent class kernels") + " (%d items)" % len(items),
                        "bound": "hbm",
                        "achieved": kbytes / (ms_kernel / 1e3) / 1e9, "unit": "GB/s", "bytes": kbytes},
           "configs": {"%s/%s" % (items_g["name"], f): batch.describe(k)
                       for k, (items_g, f) in enumerate((g, f) for g in groups for f in MIXED_FORMS)}}
    if ref is not None:
        errs = {}
        for gi, g in enumerate(groups):
            idx, refs = ref[gi]
            it = torch.from_numpy(idx).cuda()
            for fi, f in enumerate(MIXED_FORMS):
                Kref, Kabs = refs[f]
                K = batch.outputs[gi * len(MIXED_FORMS) + fi][it].double().cpu().numpy()
                e = float((np.sqrt(((K - Kref) ** 2).sum((1, 2))) / np.sqrt((Kabs ** 2).sum((1, 2)))).max())
                errs["%s/%s" % (g["name"], f)] = e
        out["rel_err_vs_abs_terms"] = errs
    batch.free()
    mats_p.free()
    mats_l.free()
    ctx.close()
    return out


def paths_measure(device, flush, steps, warmup, scale=1.0, groups=""):
    """Each mixed-mesh item's element matrices (FP32 from a stored FP32 geometry) on
    the CUDA-core path ("f32") and, where a tensor-core kernel covers the item, on the
    TF32x3 tensor-core path: the median of `steps` CUDA-event timings after `warmup`
    untimed calls, L2 flushed before each -- the choice the batch autotuner makes."""
    import torch

    from paper_2107_04121_gb300 import fe
    ctx, grps, forms = mixed_setup(scale, device)
    want = {g for g in groups.split(",") if g}
    out = {}
    for g in grps:
        if want and g["name"] not in want:
            continue
        for fname in MIXED_FORMS:
            f, mat, E = forms[fname], g["mats"][fname], g["mesh"].n_elems
            n = g["geom"].N * (3 if fname == "elasticity" else 1)
            K = torch.empty((E, n, n), dtype=torch.float32, device="cuda")
            row = {}
            for prec in ("f32", "tf32x3"):
                try:
                    fe.eval_matrix(ctx, f, g["geom"], [mat, None, None], prec, out=K)
                except fe.FEError:
                    continue
                for _ in range(warmup):
                    fe.eval_matrix(ctx, f, g["geom"], [mat, None, None], prec, out=K)
                ts = []
                for _ in range(steps):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    fe.eval_matrix(ctx, f, g["geom"], [mat, None, None], prec, out=K)
                    b.record()
                    b.synchronize()
                    ts.append(a.elapsed_time(b))
                row["cuda_core_ms" if prec == "f32" else "tensor_core_ms"] = statistics.median(ts)
            out["%s/%s" % (g["name"], fname)] = dict(row, elements=E)
            del K
    ctx.check()
    ctx.close()
    return out


def fp64_units(device, steps=2048):
    """FP64 rates of the device from fe_diag_fp64: DFMA chains and FP64 tensor-core
    MMA chains (mma.sync m8n8k4), one CTA of W warps per SM, ILP independent chains
    per lane; FMAs per clock per SM at the sampled clock, and TFLOP/s."""
    import torch

    from paper_2107_04121_gb300 import fe
    ctx = fe.Context(device)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    out = torch.empty(sms * 32 * 32, dtype=torch.float64, device="cuda")
    rows = []
    with ClockSampler(device) as clk:
        for kind, name, per_step in ((0, "dfma", 32), (1, "dmma_m8n8k4", 256)):
            for warps, ilp in ((1, 1), (2, 1), (4, 1), (8, 1), (16, 1), (4, 2), (4, 4), (8, 4)):
                fe.diag_fp64(ctx, kind, warps, ilp, steps, out)  # warm-up
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fe.diag_fp64(ctx, kind, warps, ilp, steps, out)
                b.record()
                b.synchronize()
                ms = a.elapsed_time(b)
                fmas = sms * warps * ilp * steps * per_step
                rows.append({"kind": name, "warps_per_sm": warps, "ilp": ilp, "ms": ms,
                             "tflops": 2 * fmas / (ms * 1e-3) / 1e12, "fma_per_clk_sm_at_2070": fmas / (ms * 1e-3) / sms
                             / 2.07e9})
    ctx.check()
    ctx.close()
    best = {k: max(r["tflops"] for r in rows if r["kind"] == k) for k in ("dfma", "dmma_m8n8k4")}
    return {"rows": rows, "best_tflops": best, "clocks": clk.summary()}


# ---- CPU oracle (baseline / reference arm) ------------------------------------------------

def oracle_step(mesh, lam, mu, u, n_elems):
    """One oracle step (geometry, K_e, r_e, assembly) on the first n_elems elements."""
    import oracle
    ref = oracle.RefElement(2, 3)
    conn = np.ascontiguousarray(mesh.conn[:n_elems])
    wdetJ, G, _ = oracle.geometry(mesh.coords, conn, ref)
    D = oracle.lame_to_D(lam[:n_elems], mu[:n_elems])
    oracle.matrix_elasticity(wdetJ, G, D)
    r = oracle.residual_elasticity(conn, wdetJ, G, D, u)
    oracle.assemble(conn, r, mesh.n_nodes, 3)


def cpu_model():
    """The host CPU's model string (x86 'model name', else Arm implementer/part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    for key in ("model name", "Model"):
        for line in info:
            if line.startswith(key) and ":" in line:
                return line.split(":", 1)[1].strip()
    parts = {}
    for line in info:
        if ":" in line:
            k, v = (x.strip() for x in line.split(":", 1))
            if k in ("CPU implementer", "CPU part") and k not in parts:
                parts[k] = v
    return ("Arm implementer %s part %s" % (parts.get("CPU implementer"), parts.get("CPU part"))) if parts else "unknown"


def cpu_baseline(n, min_seconds=10.0):
    """The CPU-baseline leg: the FP64 oracle timed on the host cores over whole
    steps of the full workload, repeated until at least `min_seconds` have passed
    (the sample), and the oracle references of the convection (64 sampled
    elements), adjoint and mixed-mesh workloads.  The metric workload's outputs are
    checked on every element by every_element_errors, after the GPU runs."""
    import oracle
    from paper_2107_04121_gb300 import meshgen
    mesh, lam, mu, u = meshgen.elasticity_q2_cube(n, seed=1)
    oracle_step(mesh, lam, mu, u, 64)
    reps, t, per = 0, time.perf_counter(), []
    while True:
        t1 = time.perf_counter()
        oracle_step(mesh, lam, mu, u, mesh.n_elems)
        per.append(time.perf_counter() - t1)
        reps += 1
        dt = time.perf_counter() - t
        if dt >= min_seconds:
            break
    cores = oracle.num_threads()
    # the paper's statistic T^ww: the mean without the worst repetition
    tww = statistics.mean(sorted(per)[:-1]) if len(per) > 1 else per[0]
    base = {"value": reps * mesh.n_elems / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d full oracle steps over all %d elements (FP64 geometry, K_e, r_e, assembly), %.1f s"
                      % (reps, mesh.n_elems, dt),
            "step_s": {"median": statistics.median(per), "mean_without_worst": tww},
            "cpu": cpu_model(), "affinity_cores": len(os.sched_getaffinity(0))}
    # one core, on a sixteenth of the elements
    n1 = max(1, mesh.n_elems // 16)
    oracle.set_num_threads(1)
    try:
        t1 = time.perf_counter()
        oracle_step(mesh, lam, mu, u, n1)
        d1 = time.perf_counter() - t1
    finally:
        oracle.set_num_threads(cores)
    base["single_thread"] = {"value": n1 / d1, "unit": UNIT, "sample": "one step over the first %d elements, %.1f s"
                                                                        % (n1, d1)}
    return base, (convect_reference(CONVECT_N), adjoint_reference(ADJOINT_N), mixed_reference())


def mixed_reference(scale=1.0, per_group=16):
    """CPU-baseline leg, mixed mesh: the oracle's matrices of the three forms
    on sampled elements of every group, with the sums of absolute terms."""
    import oracle
    from paper_2107_04121_gb300 import meshgen
    out = []
    for name, mesh in meshgen.mixed_mesh_groups(scale, seed=2):
        p = int(name[1])
        ref = oracle.RefTet(p, p) if name[0] == "P" else oracle.RefElement(p, p + 1)
        rng = np.random.default_rng(100 + p + (10 if name[0] == "P" else 0))
        coef = rng.uniform(0.5, 2.0, mesh.n_elems)
        lam, mu = rng.uniform(0.5, 2.0, mesh.n_elems), rng.uniform(0.2, 1.0, mesh.n_elems)
        E = mesh.n_elems
        idx = np.unique(np.concatenate([[0, E - 1], np.random.default_rng(11).choice(E, per_group, replace=False)]))
        wdetJ, G, _ = oracle.geometry(mesh.coords, mesh.conn[idx], ref)
        aw, aG = np.abs(wdetJ), np.abs(G)
        D = oracle.lame_to_D(lam[idx], mu[idx])
        out.append((idx, {"laplace": (oracle.matrix_laplace(wdetJ, G, coef[idx]),
                                      oracle.matrix_laplace(aw, aG, coef[idx])),
                          "mass": (oracle.matrix_mass(wdetJ, ref.phi, 1, coef[idx]),
                                   oracle.matrix_mass(aw, np.abs(ref.phi), 1, coef[idx])),
                          "elasticity": (oracle.matrix_elasticity(wdetJ, G, D),
                                         oracle.matrix_elasticity(aw, aG, np.abs(D)))}))
    return out


def adjoint_reference(n):
    """CPU-baseline leg, adjoint workload: the oracle's J and gradient."""
    import oracle
    from paper_2107_04121_gb300 import meshgen
    mesh, lam, mu, u = meshgen.elasticity_q2_cube(n, seed=4, perturb=0.1)
    return oracle.elasticity_objective_gradient(mesh.coords, mesh.conn, oracle.RefElement(2, 3), lam, mu, u)


def convect_reference(n):
    """CPU-baseline leg, convection workload: the oracle's K_e(u) and r_e(u) on 64
    sampled elements (first, last, 62 seeded)."""
    import oracle
    from paper_2107_04121_gb300 import meshgen
    mesh, u = meshgen.convect_q2_cube(n, seed=3)
    E = mesh.n_elems
    rng = np.random.default_rng(9)
    idx = np.unique(np.concatenate([[0, E - 1], rng.choice(E, min(62, E), replace=False)]))
    ref = oracle.RefElement(2, 3)
    conn = mesh.conn[idx]
    wdetJ, G, _ = oracle.geometry(mesh.coords, conn, ref)
    return (idx, oracle.matrix_convect(conn, wdetJ, ref.phi, G, u), oracle.residual_convect(conn, wdetJ, ref.phi, G, u))


def cpu_info():
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return model


def workload_description(n, E):
    """The metric's workload, as both arms name it in their `config`."""
    return ("Q2 linear elasticity, %d^3 = %d hexes (27 nodes, 27 Gauss points), +-0.15h interior "
            "perturbation seed 1, per-element Lame lambda~U[0.5,2], mu~U[0.2,1], u~N(0,1); step = FP64 "
            "geometry + r_e + K_e (81x81) + assembly" % (n, E))


def run_reference(args, ws, rank):
    """The reference arm: the FP64 oracle over whole steps of the metric's workload
    (every element: geometry, K_e, r_e, assembly) on the host cores.  Warm-up steps
    run over the first 4,096 elements (untimed); each timed step covers all of them."""
    if rank != 0:
        return
    import oracle
    from paper_2107_04121_gb300 import meshgen
    mesh, lam, mu, u = meshgen.elasticity_q2_cube(args.n, seed=1)
    E = mesh.n_elems
    for _ in range(args.warmup):
        oracle_step(mesh, lam, mu, u, min(4096, E))
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle_step(mesh, lam, mu, u, E)
        ts.append(time.perf_counter() - t)
    ms = 1e3 * sum(ts) / len(ts)
    value = E / (ms / 1e3)
    cores = oracle.num_threads()
    desc = ("%d whole steps over all %d elements, FP64 nested-loop oracle (geometry, K_e, r_e, assembly), "
            "%d OpenMP threads, %s" % (args.steps, E, cores, cpu_info()))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_description(args.n, E), "elements": E},
            "contraction": "f64 (oracle)",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- main ------------------------------------------------------------------------------------

def main():
    args = parse_args()
    if args.impl == "reference":
        # the oracle arm runs on rank 0's host cores only; other ranks exit at once
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        return
    ws, rank, local = dist_setup(args)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    if args.workload == "fp64units":
        if rank == 0:
            print(json.dumps({"workload": "fp64units", **fp64_units(local)}), flush=True)
        return
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    if args.workload == "paths":
        if rank == 0:
            print(json.dumps({"workload": "paths", "steps": args.steps, "warmup": args.warmup,
                              "items": paths_measure(local, flush, max(args.steps, 1), args.warmup, args.scale,
                                                     args.groups)}), flush=True)
        return
    if args.workload in ("convection", "mixed"):
        if args.workload == "convection":
            res = convect_measure(args.n, local, ws, flush, None, hbm_peak, args.steps, args.warmup)
        else:
            res = mixed_measure(local, flush, None, args.steps, args.warmup, args.scale)
            res["roofline"].update({"peak": hbm_peak, "frac": res["roofline"]["achieved"] / hbm_peak})
        if rank == 0:
            print(json.dumps({"workload": args.workload, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                              **res}), flush=True)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    # the oracle's OpenMP threads must not compete with the timed GPU region:
    # time the CPU baseline first (rank 0, N = 1 only)
    cpu, cv_ref, ad_ref, mx_ref = None, None, None, None
    if rank == 0 and ws == 1 and not args.skip_extras:
        cpu, (cv_ref, ad_ref, mx_ref) = cpu_baseline(args.n)

    wl = Workload(args.n, local)
    ladder, errs, prec_note = None, None, None
    prec = args.prec
    if prec == "auto":
        ladder = precision_ladder(wl, flush)
    if cpu is not None:
        # every element of every precision's step against the oracle (the FP64
        # path's too), then the fastest rung within 1e-5 on all of them
        checked = (LADDER if ladder is not None else [prec]) + ["f64"]
        for p in checked:
            if p not in wl.bufs:
                wl.step(p)
        wl.ctx.check()
        errs = every_element_errors(wl, checked)
        errs["elements_checked"] = wl.E
        if ladder is not None:
            for p in LADDER:
                ladder[p].update({"rel_err_K": errs["K_" + p], "rel_err_r": errs["r_" + p]})
            ok = [p for p in LADDER if ladder[p]["rel_err_K"] <= 1e-5 and ladder[p]["rel_err_r"] <= 1e-5]
            if ok:
                prec = min(ok, key=lambda p: ladder[p]["matrix_ms"])
            else:
                prec = "f32"
                prec_note = "no contraction precision met 1e-5 on every element; the f32 rung is timed"
                print("bench: " + prec_note, file=sys.stderr, flush=True)
    elif prec == "auto":
        prec = DEFAULT_MIXED  # no oracle on this rank: the precision the N = 1 run selects
    for p in list(wl.bufs):
        if p != prec:
            wl.drop(p)
    with ClockSampler(local) as clk:
        step_ms, mat_ms, parts = timed_steps(wl, prec, args.steps, args.warmup, ws, flush)
    value, ms_per_step = job_rate(step_ms, wl.E, args.steps, ws)
    mat_avg = sum(mat_ms) / len(mat_ms)
    fused = wl.matrix_first(prec)
    mat_bytes = MATRIX_GEO_BYTES_PER_ELEM if fused else (MATRIX_BYTES_PER_ELEM_F64 if prec == "f64"
                                                         else MATRIX_BYTES_PER_ELEM_F32)
    bytes_alg = wl.E * mat_bytes
    achieved = bytes_alg / (mat_avg / 1e3) / 1e9
    kname = ("k_matrix_tc<%s> with its geometry warps (fe_eval_matrix computing the deferred FP64 geometry)" % prec
             if fused else "k_matrix (fe_eval_matrix, %s)" % prec)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec != "f64" else "f64", "data": "synthetic",
        "config": {"workload": workload_description(args.n, wl.E), "elements": wl.E,
                   "l2": "flushed between timed steps (512 MiB write)", "parallelism": "replicas"},
        "contraction": prec, "geometry_dtype": "f64",
        "roofline": {"kernel": kname, "bound": "hbm", "achieved": achieved,
                     "peak": hbm_peak, "peak_source": peak_src, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "traffic": MEASURED_TRAFFIC_48.get("matrix_geo_" + prec) if (args.n == 48 and fused) else None,
                     "bytes_per_elem": mat_bytes, "avg_ms": mat_avg},
        "gpu_launches": kernels_per_step(prec) * args.steps,
        "step_parts_ms": parts,
    }
    line["clocks"] = clk.summary()
    if prec != "f64":
        # FP64 geometry: lane-instructions per element against the issue peak of the
        # FP64 units (2 lanes per clock per SM) at the sampled clock, over the time of
        # the kernel that computes it (the matrix kernel's geometry warps, or the
        # geometry + residual kernel)
        t_geo = (parts["matrix_with_geometry"] if fused else parts["geometry_and_residual"]) / 1e3
        mhz = line["clocks"].get("sm_mhz") or line["clocks"].get("sm_max_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        issue_peak = FP64_LANES_PER_CLK_SM * sms * mhz * 1e6 / 1e9
        issue = wl.E * GEOMETRY_FP64_INSTR_PER_ELEM_Q2 / t_geo / 1e9
        line["roofline_fp64_geometry"] = {
            "kernel": kname if fused else "k_residual_geo (FP64 geometry + r_e, f32)", "bound": "fp64",
            "instructions_per_elem": GEOMETRY_FP64_INSTR_PER_ELEM_Q2, "achieved": issue, "peak": issue_peak,
            "unit": "G FP64 lane-instructions/s", "frac": issue / issue_peak,
            "peak_basis": "%d FP64 lanes per clock per SM (measured) x %d SMs x median SM clock %.0f MHz"
                          % (FP64_LANES_PER_CLK_SM, sms, mhz),
            "avg_ms": t_geo * 1e3}
        # the whole step against its floor: the larger of its algorithmic bytes at the
        # HBM copy rate and its FP64 geometry at the FP64 issue peak
        asm_bytes = 81 * 4 + Q2_N * 4 + (wl.mesh.n_nodes + 1) * 4 / wl.E + wl.mesh.n_nodes * 3 * 4 / wl.E
        step_bytes = MATRIX_GEO_BYTES_PER_ELEM + RESIDUAL_BYTES_PER_ELEM + asm_bytes
        t_hbm = wl.E * step_bytes / (hbm_peak * 1e9) * 1e3
        t_fp64 = wl.E * GEOMETRY_FP64_INSTR_PER_ELEM_Q2 / (issue_peak * 1e9) * 1e3
        floor = max(t_hbm, t_fp64)
        line["roofline_step"] = {
            "bound": "hbm" if t_hbm >= t_fp64 else "fp64", "floor_ms": floor, "ms_per_step": ms_per_step,
            "frac": floor / ms_per_step, "bytes_per_elem": step_bytes, "hbm_ms": t_hbm, "fp64_ms": t_fp64,
            "basis": "step bytes (matrix with geometry, residual, assembly) / measured HBM copy rate vs FP64 "
                     "geometry lane-instructions / FP64 issue peak; frac = floor / ms_per_step"}
    if ladder is not None:
        line["precision_ladder"] = ladder
    if prec_note:
        line["precision_note"] = prec_note
    if not args.skip_extras and prec != "f64":
        # the step's geometry variants, timed alone: the tensor-core kernel computing
        # it, the residual kernel computing it, and the geometry kernel followed by
        # the residual and the matrix on the stored float32 copy
        K, r, g = wl.outputs(prec)
        g32, gd = wl.geoms["f32"], wl.geoms["f32d"]
        mat_args = [wl.mat, None, None]
        res_args = [wl.mat, None, wl.u32]
        def fused_matrix():
            gd.update()
            wl.fe.eval_matrix(wl.ctx, wl.form, gd, mat_args, prec, out=K)
        def fused_residual():
            gd.update()
            wl.fe.eval_residual(wl.ctx, wl.form, gd, res_args, prec, out=r)
        t_fm = time_call(wl, flush, fused_matrix) if wl.matrix_first(prec) else None
        t_fr = time_call(wl, flush, fused_residual)
        t_geo = time_call(wl, flush, lambda: g32.update())
        t_res = time_call(wl, flush, lambda: wl.fe.eval_residual(wl.ctx, wl.form, g32, res_args, prec, out=r))
        t_mat = time_call(wl, flush, lambda: wl.fe.eval_matrix(wl.ctx, wl.form, g32, mat_args, prec, out=K))
        line["geometry_variants_ms"] = {
            "matrix_kernel_computing_geometry": t_fm, "residual_kernel_computing_geometry": t_fr,
            "stored_geometry": {"geometry": t_geo, "residual": t_res, "matrix": t_mat},
            "steps_without_assembly": {"matrix_first": None if t_fm is None else t_fm + t_res,
                                       "residual_first": t_fr + t_mat, "geometry_first": t_geo + t_res + t_mat}}
    if not args.skip_extras:
        wl.drop(prec)
        # plain FP64 path, same step
        f64_steps = 3
        s64, m64, p64 = timed_steps(wl, "f64", f64_steps, 1, ws, flush)
        t64 = max_over_ranks(sum(s64), ws)
        line["fp64_path"] = {"value": ws * wl.E * f64_steps / (t64 / 1e3), "unit": UNIT,
                             "ms_per_step": t64 / f64_steps, "matrix_ms": sum(m64) / len(m64), "parts_ms": p64}
        wl.drop("f64")
        if errs is not None:
            line["rel_err"] = errs
        line["speedup_vs_fp64_path"] = value / line["fp64_path"]["value"]
        line["e2e"] = e2e_measure(wl, prec, 5, ws)
        # the Navier-Stokes convection workload (Eq. fe2, fe4), same device
        for p in list(wl.bufs):
            wl.drop(p)
        line["convective"] = convect_measure(CONVECT_N, local, ws, flush, cv_ref, hbm_peak)
        line["adjoint"] = adjoint_measure(ADJOINT_N, local, flush, ad_ref)
        line["mixed"] = mixed_measure(local, flush, mx_ref)
        line["mixed"]["roofline"].update({"peak": hbm_peak, "frac": line["mixed"]["roofline"]["achieved"] / hbm_peak})
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
