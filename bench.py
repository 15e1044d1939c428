#!/usr/bin/env python
"""Benchmark: finite element assembly throughput on GB300.

One step = one pass of the assembly hot path over the workload: per-element
Jacobians, local matrices and load vectors by quadrature, and the
deterministic scatter into the CSR values and the load vector (the CSR
pattern is built once beforehand and reported separately).  Default
workload, the largest single-GPU configuration: P1 linear elasticity on the
128^3 Kuhn cube mesh (12,582,912 tets, 6,440,067 dofs, 286,222,473
nonzeros), Lame parameters uniform in [0.5, 2] per element, body force
(0, 0, -1), FP64, with the chunked fixed-point scatter.  The other
configurations (P2 diffusion + mass 64^3, P1 kappa-diffusion 96^3 and its
adjoint, the 256-mesh batch, P1 Poisson 8^3) and the other forms are timed
in the same run, each with its own roofline entry.

Prints one JSON line.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

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

import numpy as np  # noqa: E402

from paper_1802_03433_gb300 import meshgen as mg  # noqa: E402

# Nominal FP64 peak: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (1.26 TFLOP/s);
# the roofline uses the rate fea_diag_fp64_rate measures on the device at the
# start of every run and reports the nominal fraction beside it.
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# The dominant kernel of each workload: FP64 flop per element counted in FP64
# terms ("equivalent": the element formulas as FP64 operations, DFMA = 2),
# the FP64 flop the kernel executes per element (ncu SASS counters: 2 DFMA +
# DADD + DMUL; lower where exact integer arithmetic replaced FP64 work), and
# its DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum,
# one capture; the captures are summarised under profiles/).  fp64_instr is
# the FP64 instructions (DFMA + DADD + DMUL, ncu SASS thread counts) the
# kernel executes per element: the FP64 pipe issues one of them per slot
# whatever its kind, so their rate against the measured DFMA instruction
# rate is how busy that pipe is kept.
KERNELS = {
    # chunked scatter: the element arithmetic plus the bound of phase A;
    # counters of the 64^3 capture (93 DFMA + 25 DADD + 99 DMUL = 217 FP64
    # instructions, 310 flop per element); DRAM bytes of one 128^3 launch
    # (one-pass launch list) and of one 64^3 launch (full capture)
    "p1_elast_128": dict(kernel="k_elast_chunk (element arithmetic + fixed-point accumulation per chunk)",
                         flop_equiv=310.0, flop_exec=310.0, fp64_instr=217.0, traffic=1631.0e6 + 3187.9e6,
                         profile="profiles/element_chunk_kernel_p1_elast.md"),
    "p1_elast_64": dict(kernel="k_elast_chunk", flop_equiv=310.0, flop_exec=310.0, fp64_instr=217.0,
                        traffic=199.4e6 + 354.9e6, profile="profiles/element_chunk_kernel_p1_elast.md"),
    # P2: matrix warps + load warps; 375 = the formulas in FP64 (150 DFMA +
    # 26 DADD + 49 DMUL); executed 31 DFMA + 30 DADD + 43 DMUL (the 136 FMA
    # terms of the entries are exact 64-bit integer sums)
    "p2_diffmass_64": dict(kernel="k_elem_roles (P2 element, FP64)", flop_equiv=375.0, flop_exec=135.0, fp64_instr=104.0,
                           traffic=148.8e6 + 1967.0e6, profile="profiles/element_kernel_p2_diffmass_64.md"),
    # P1: 27 DFMA + 25 DADD + 32 DMUL
    "p1_kappa_96": dict(kernel="k_elem_scalar (P1 element, FP64)", flop_equiv=111.0, flop_exec=111.0, fp64_instr=84.0,
                        traffic=238.9e6 + 792.2e6, profile="profiles/element_kernel_p1_kappa_96.md"),
    "p1_poisson_8": dict(kernel="k_elem_scalar (P1 element, FP64)", flop_equiv=111.0, flop_exec=111.0, fp64_instr=84.0,
                         traffic=None, profile=None),
    "adjoint_96": dict(kernel="k_adjoint (P1 backward, FP64)", flop_equiv=370.0, flop_exec=370.0, fp64_instr=250.0,
                       traffic=438.0e6 + 672.1e6, profile="profiles/adjoint_kernel_p1_kappa_96.md"),
    "paper_2d": dict(kernel="k_elem_tri (P1 triangle element, FP64)", flop_equiv=191.0, flop_exec=191.0, fp64_instr=127.0,
                     traffic=268.5e6 + 950.7e6, profile="profiles/element_kernel_paper_2d.md"),
}

METRIC = "elements/s assembled into CSR and % of HBM roofline, plain vs chosen forms"

WORKLOADS = {
    "p1_elast_128": dict(kind="elasticity", n=128),
    "p2_diffmass_64": dict(kind="p2_diffmass", n=64),
    "p1_poisson_8": dict(kind="p1_poisson", n=8),
    "p1_elast_64": dict(kind="elasticity", n=64),     # small case of the same kernel, for multi-pass captures
    "p1_kappa_96": dict(kind="p1_kappa", n=96),
}


def mixed_error(torch, mesh, d, ref_vals, vals, ref_rhs, rhs):
    """Row-scaled error of the mixed-precision result against the FP64 result
    of the same run (max over rows of max |dA| / max |A_fp64| in the row; rhs
    scaled by its max), computed on the device.  The FP64 path is within 1e-12
    of the oracle, so this is the mixed path's error against the oracle to
    that accuracy."""
    rp, _ = mesh.pattern_tensors(d["order"], d["ndpn"])
    counts = torch.diff(rp.long())
    rows = torch.repeat_interleave(torch.arange(counts.numel(), device=rp.device), counts)
    nnz = rows.numel()
    diff = (vals[:nnz] - ref_vals[:nnz]).abs()
    scale = torch.zeros(counts.numel(), dtype=torch.float64, device=rp.device)
    scale.scatter_reduce_(0, rows, ref_vals[:nnz].abs(), reduce="amax")
    worst = torch.zeros_like(scale).scatter_reduce_(0, rows, diff, reduce="amax")
    row_err = torch.where(scale > 0, worst / torch.where(scale > 0, scale, torch.ones_like(scale)), worst)
    rhs_err = (rhs - ref_rhs).abs().max() / ref_rhs.abs().max().clamp_min(1e-300)
    return {"values_row_scaled": float(row_err.max()), "rhs_scaled": float(rhs_err)}


def algorithmic_bytes(kind, E, N, ndof, nnz):
    """Inputs read once + outputs written once: coords 24 B/node, the element
    -> dof table (16 B/element for P1, 40 B for the ten P2 dofs),
    coefficients 8 B per field per element, values 8 B/nnz, rhs 8 B/dof."""
    coef = {"p1_poisson": 0, "p1_kappa": 8, "p2_diffmass": 8, "elasticity": 16}[kind]
    table = 40 if kind == "p2_diffmass" else 16
    return 24 * N + table * E + coef * E + 8 * nnz + 8 * ndof


def roofline_block(key, E, kernel_ms, fp64_peak_tflops, note=None):
    """Roofline entry of the dominant (FP64-bound) kernel of a workload:
    achieved = FP64 flop per element x elements / the kernel's CUDA-event
    time, against the FP64 rate measured on this device (frac) and the
    nominal one (frac_nominal); the same for the FP64 flop the kernel
    actually executes."""
    k = KERNELS.get(key)
    if k is None or not kernel_ms:
        return None
    ach = k["flop_equiv"] * E / (kernel_ms / 1e3) / 1e12
    exe = k["flop_exec"] * E / (kernel_ms / 1e3) / 1e12
    out = {"kernel": k["kernel"], "bound": "alu", "achieved": ach, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
           "frac": ach / fp64_peak_tflops, "peak_kind": "FP64 FMA rate measured on this GPU (fea_diag_fp64_rate)",
           "frac_nominal": ach / FP64_NOMINAL_TFLOPS, "flop_per_element": k["flop_equiv"],
           "executed": {"flop_per_element": k["flop_exec"], "achieved": exe, "frac": exe / fp64_peak_tflops},
           "kernel_ms": kernel_ms, "traffic": k["traffic"], "profile": k["profile"]}
    if k.get("fp64_instr"):
        # FP64 pipe issue: instructions per second against the measured DFMA
        # instruction rate (the measured flop rate / 2)
        ips = k["fp64_instr"] * E / (kernel_ms / 1e3) / 1e9
        peak_ips = fp64_peak_tflops * 1e3 / 2
        nominal_ips = FP64_NOMINAL_TFLOPS * 1e3 / 2  # 2 FP64 instructions per SM and clock
        out["fp64_pipe"] = {"instr_per_element": k["fp64_instr"], "achieved_ginstr_s": ips,
                            "peak_ginstr_s": peak_ips, "frac": ips / peak_ips,
                            "peak_nominal_ginstr_s": nominal_ips, "frac_nominal": ips / nominal_ips}
    if note:
        out["note"] = note
    return out


def hbm_block(alg_bytes, step_ms):
    gbs = alg_bytes / (step_ms / 1e3) / 1e9
    return {"algorithmic_bytes": alg_bytes, "achieved_gbs": gbs, "peak_gbs": _hbm_peak(), "frac": gbs / _hbm_peak()}


def make_inputs(kind, n, seed=0):
    coords, tets, rng = mg.make_cube(n, 0.2, seed)
    E = tets.shape[1]
    d = dict(coords=coords, tets=tets, kind=kind, n=n)
    if kind == "p1_poisson":
        d.update(order=1, ndpn=1, form=0, mass=0.0, kappa=None, f_kind=2, f_param=(mg.SIN_AMP,), npts=4)
    elif kind == "p1_kappa":
        d.update(order=1, ndpn=1, form=0, mass=0.0, kappa=mg.lognormal(rng, E), f_kind=2,
                 f_param=(mg.SIN_AMP,), npts=4)
    elif kind == "p2_diffmass":
        d.update(order=2, ndpn=1, form=1, mass=1.0, kappa=mg.lognormal(rng, E), f_kind=2,
                 f_param=(mg.SIN_AMP,), npts=11)
    elif kind == "elasticity":
        lam, mu = mg.lame(rng, E)
        d.update(order=1, ndpn=3, form=2, mass=0.0, lam=lam, mu=mu, f_kind=1, f_param=(0.0, 0.0, -1.0), npts=4)
    return d


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(",") for l in self.f.read().splitlines() if l.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for nm, v in zip(names, r[4:8]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device="cpu"):
    """The largest of every rank's value (the job finishes with its slowest
    rank); a plain float without an initialised process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


# Clock-event reasons that reject a timed region (sw_power_cap is kept and
# noted: a dense kernel on a 1.4 kW part may run at the power cap).
THROTTLE_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def throttled(clk):
    """Whether the clock record of a timed region rejects its number."""
    return bool(clk) and any(r in clk.get("reasons", ()) for r in THROTTLE_REASONS)


def weak_scaling_value(world_size, units_per_rank, steps, total_ms):
    """Whole-job throughput: every rank processes its own units each step."""
    return world_size * units_per_rank * steps / (total_ms / 1e3)


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        from paper_1802_03433_gb300 import build_lib
        build_lib.build()
    if ws > 1:
        dist.barrier()
    from paper_1802_03433_gb300 import fea

    wl = WORKLOADS[args.workload]
    # several GPUs: a P1 mesh is split by rows (fea_partition: each rank owns a
    # z-slab of nodes and assembles its elements plus the ghost layer, with no
    # exchange; strong scaling of one mesh); otherwise (P2, or --replicas)
    # every rank assembles its own copy of the workload (weak scaling)
    partitioned = ws > 1 and not args.replicas and wl["kind"] != "p2_diffmass"
    d = make_inputs(wl["kind"], wl["n"], seed=args.seed + (0 if partitioned else rank))
    E_total = d["tets"].shape[1]
    if partitioned:
        part = fea.fea_partition(d["tets"], d["coords"].shape[1], ws, rank)
        d = dict(d, coords=np.ascontiguousarray(d["coords"][:, part["nodes"]]), tets=part["sub_tets"])
        for key in ("kappa", "lam", "mu"):
            if d.get(key) is not None:
                d[key] = np.ascontiguousarray(d[key][part["elems"]])
    dev = torch.device("cuda", local)
    E = d["tets"].shape[1]
    N = d["coords"].shape[1]

    # the FP64 peak the rooflines divide by, measured on this device
    fp64_peak = fea.fea_diag_fp64_rate() / 1e12
    mesh = fea.Mesh(d["coords"], d["tets"], device=dev)
    fea.fea_mesh_set_scatter(mesh.h, args.scatter)
    fea.fea_mesh_set_stages(mesh.h, args.stages)
    if args.scatter_classes >= 0:
        fea.fea_mesh_set_scatter_classes(mesh.h, args.scatter_classes)
    if args.load_split >= 0:
        fea.fea_mesh_set_load_split(mesh.h, args.load_split)
    if args.scatter_stages > 0:
        fea.fea_mesh_set_scatter_stages(mesh.h, args.scatter_stages)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ndof, nnz = mesh.pattern(d["order"], d["ndpn"])
    pattern_ms = (time.perf_counter() - t0) * 1e3

    keep = []
    if d["form"] == 2:
        lam = torch.as_tensor(d["lam"], device=dev)
        mu = torch.as_tensor(d["mu"], device=dev)
        keep += [lam, mu]
        coeffs = fea.make_coeffs(lam=lam, mu=mu, f_kind=d["f_kind"], f_param=d["f_param"])
    else:
        kap = None if d["kappa"] is None else torch.as_tensor(d["kappa"], device=dev)
        keep.append(kap)
        coeffs = fea.make_coeffs(kappa=kap, f_kind=d["f_kind"], f_param=d["f_param"])
    form = fea.make_form(d["form"], d["order"], d["mass"])
    values = torch.empty(nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(ndof, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > L2
    fea.fea_profile_enable(mesh.h, True)

    def timed_loop(prec, steps, warmup, clocks=None):
        quad = fea.make_quadrature(d["npts"], prec)
        for _ in range(warmup):
            fea.fea_assemble(mesh.h, form, coeffs, quad, values, rhs)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
            time.sleep(0.3)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        phase = []
        for k in range(steps):
            flush.fill_(k)
            evs[k][0].record()
            fea.fea_assemble(mesh.h, form, coeffs, quad, values, rhs)
            evs[k][1].record()
            phase.append(fea.fea_profile_last(mesh.h))
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        if ws > 1:
            dist.barrier()
        mesh.check()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        return max_over_ranks(sum(step_ms), dev), step_ms, phase, clk

    clocks = ClockSampler(local) if rank == 0 else None
    total_ms, step_ms, phase, clk = timed_loop(fea.FEA_FP64, args.steps, args.warmup, clocks)
    # a slowdown seen during the timed region rejects it: measure once more
    # (every rank takes the same decision; the loop has barriers)
    if max_over_ranks(1.0 if throttled(clk) else 0.0, dev) > 0.0:
        first = clk
        total_ms, step_ms, phase, clk = timed_loop(fea.FEA_FP64, args.steps, args.warmup, clocks)
        if clk is not None:
            clk = dict(clk, remeasured_after=first.get("reasons", []) if first else [])
    value = (E_total * args.steps / (total_ms / 1e3)) if partitioned else weak_scaling_value(ws, E, args.steps,
                                                                                              total_ms)
    elem_ms = statistics.mean(p[0] for p in phase)
    scat_ms = statistics.mean(p[1] for p in phase)

    # mixed-precision form on the same GPU and workload
    forms = {"fp64": {"value": value, "ms_per_step": total_ms / args.steps, "elem_ms": elem_ms,
                      "scatter_ms": scat_ms}}
    def want(name):
        return not args.no_forms and (args.forms == "all" or name in args.forms.split(","))

    if want("mixed"):
        ref_vals, ref_rhs = values.clone(), rhs.clone()  # the FP64 result of the loop above
        m_total, _, m_phase, _ = timed_loop(fea.FEA_MIXED, max(3, args.steps // 2), args.warmup)
        ms = m_total / max(3, args.steps // 2)
        forms["mixed"] = {"value": ws * E / (ms / 1e3), "ms_per_step": ms,
                          "elem_ms": statistics.mean(p[0] for p in m_phase),
                          "scatter_ms": statistics.mean(p[1] for p in m_phase),
                          "error_vs_fp64": mixed_error(torch, mesh, d, ref_vals, values, ref_rhs, rhs)}

    small = max(3, args.steps // 4)
    if want("atomic_alg1"):
        # the paper's sparse Algorithm 1 on the same workload: row search +
        # global FP64 atomicAdd (no scratch, no reproducibility)
        quad = fea.make_quadrature(d["npts"], fea.FEA_FP64)
        for _ in range(args.warmup):
            fea.fea_assemble_atomic(mesh.h, form, coeffs, quad, values, rhs)
        torch.cuda.synchronize()
        at, runs = 0.0, []
        steps_a = max(3, args.steps // 2)
        for k in range(steps_a):
            flush.fill_(k)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fea.fea_assemble_atomic(mesh.h, form, coeffs, quad, values, rhs)
            b.record()
            torch.cuda.synchronize()
            at += a.elapsed_time(b)
            if k < 2:
                runs.append(values.clone())
        at = max_over_ranks(at, dev)
        forms["atomic_alg1"] = {"value": weak_scaling_value(ws, E, steps_a, at), "ms_per_step": at / steps_a,
                                "bitwise_equal_across_two_runs": bool(torch.equal(runs[0].view(torch.int64),
                                                                                  runs[1].view(torch.int64))),
                                "note": "paper's sparse Algorithm 1: global FP64 atomicAdd after a row search"}
        del runs
    if want("batched"):
        forms["batched"] = bench_batched(fea, torch, dev, small, args.warmup, flush, ws, rank)
    if want("adjoint"):
        forms["adjoint"] = bench_adjoint(fea, torch, dev, small, args.warmup, flush, fp64_peak)
    if want("local_rows") and d["form"] == 2 and args.scatter != fea.FEA_SCATTER_LOCAL_ROWS:
        # the same workload with the local-row scatter (element kernel writes
        # every local row to HBM, row-gather kernel adds them)
        fea.fea_mesh_set_scatter(mesh.h, fea.FEA_SCATTER_LOCAL_ROWS)
        l_total, _, l_phase, _ = timed_loop(fea.FEA_FP64, small, args.warmup)
        fea.fea_mesh_set_scatter(mesh.h, args.scatter)
        forms["local_rows"] = {"value": ws * E / (l_total / small / 1e3), "ms_per_step": l_total / small,
                               "elem_ms": statistics.mean(p[0] for p in l_phase),
                               "scatter_ms": statistics.mean(p[1] for p in l_phase),
                               "note": "FEA_SCATTER_LOCAL_ROWS on the same workload, FP64"}
    for name, kind, n in (("p2_diffmass_64", "p2_diffmass", 64), ("elasticity_128", "elasticity", 128),
                          ("p1_kappa_96", "p1_kappa", 96), ("p1_poisson_8", "p1_poisson", 8)):
        same = {"elasticity_128": "p1_elast_128"}.get(name, name) == args.workload
        if want(name) and not same:
            forms[name] = bench_plain(fea, torch, dev, kind, n, small, args.warmup, flush, fp64_peak)
    if want("jit"):
        forms["jit"] = bench_jit(fea, torch, dev, small, args.warmup, flush)
    if want("solve"):
        forms["solve"] = bench_solve(fea, torch, dev)
    if want("paper_2d"):
        forms["paper_2d"] = bench_paper_2d(fea, torch, dev, small, args.warmup, flush, fp64_peak)

    # end to end through the public API with host buffers: every step copies
    # its inputs (coordinates, coefficients) host -> device from pinned
    # memory, assembles, and copies the assembled values and load vector back.
    # Two mesh handles alternate on two streams, each with its own device
    # inputs, scratch and outputs, so the copies of one step overlap the
    # assembly of the next (a stream orders each handle's own steps).
    e2e = None
    if not args.no_e2e:
        pin = lambda t: t.cpu().pin_memory()  # noqa: E731
        host_in = [pin(mesh.x), pin(mesh.y), pin(mesh.z)] + [pin(t) for t in keep if t is not None]
        quad = fea.make_quadrature(d["npts"], fea.FEA_FP64)
        lanes = []
        for i in range(2):
            mi = mesh if i == 0 else fea.Mesh(d["coords"], d["tets"], device=dev)
            if i == 1:
                fea.fea_mesh_set_stages(mi.h, args.stages)
                if args.scatter_classes >= 0:
                    fea.fea_mesh_set_scatter_classes(mi.h, args.scatter_classes)
                if args.load_split >= 0:
                    fea.fea_mesh_set_load_split(mi.h, args.load_split)
                if args.scatter_stages > 0:
                    fea.fea_mesh_set_scatter_stages(mi.h, args.scatter_stages)
                mi.pattern(d["order"], d["ndpn"])
            dev_coef = [torch.empty_like(t) for t in keep if t is not None]
            if d["form"] == 2:
                co_i = fea.make_coeffs(lam=dev_coef[0], mu=dev_coef[1], f_kind=d["f_kind"], f_param=d["f_param"])
            else:
                co_i = fea.make_coeffs(kappa=dev_coef[0] if dev_coef else None, f_kind=d["f_kind"],
                                       f_param=d["f_param"])
            lanes.append(dict(
                mesh=mi, coeffs=co_i, dev_in=[mi.x, mi.y, mi.z] + dev_coef,
                values=torch.empty(nnz, dtype=torch.float64, device=dev),
                rhs=torch.empty(ndof, dtype=torch.float64, device=dev),
                hv=torch.empty(nnz, dtype=torch.float64).pin_memory(),
                hr=torch.empty(ndof, dtype=torch.float64).pin_memory(),
                stream=torch.cuda.Stream(dev)))
        steps = max(4, args.steps // 4)

        def e2e_step(k):
            ln = lanes[k % 2]
            with torch.cuda.stream(ln["stream"]):
                for h, dv in zip(host_in, ln["dev_in"]):
                    dv.copy_(h, non_blocking=True)
                fea.fea_assemble(ln["mesh"].h, form, ln["coeffs"], quad, ln["values"], ln["rhs"],
                                 stream=ln["stream"])
                ln["hv"].copy_(ln["values"], non_blocking=True)
                ln["hr"].copy_(ln["rhs"], non_blocking=True)

        for k in range(max(2, args.warmup)):
            e2e_step(k)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for ln in lanes:
            ln["stream"].wait_event(a)
        for k in range(steps):
            e2e_step(k)
        for ln in lanes:
            torch.cuda.current_stream().wait_stream(ln["stream"])
        b.record()
        torch.cuda.synchronize()
        t_ms = max_over_ranks(a.elapsed_time(b), dev)
        h2d = sum(h.numel() * h.element_size() for h in host_in)
        d2h = nnz * 8 + ndof * 8
        e2e = {"value": weak_scaling_value(ws, E, steps, t_ms), "unit": "elements/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "pipelining": "two mesh handles on two streams"}
        lanes[1]["mesh"].close()

    # roofline of the dominant kernel (the element kernel, or for elasticity
    # the chunk kernel that computes and accumulates the elements)
    roof = roofline_block(args.workload, E, elem_ms, fp64_peak)
    forms["fp64"]["roofline"] = roof

    alg = algorithmic_bytes(d["kind"], E, N, ndof, nnz)
    forms["fp64"]["hbm"] = hbm_block(alg, total_ms / args.steps)
    if "mixed" in forms:
        forms["mixed"]["hbm"] = hbm_block(alg, forms["mixed"]["ms_per_step"])
    # kernels launched per step: chunked elasticity = the chunk kernel and the
    # two reduce kernels; the local-row path = the element kernel and the
    # scatter (the bulk-copy scatter of the scalar forms splits its row tiles
    # over two launches)
    per_step = 3
    out = None
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(d["kind"])
        out = {
            "metric": METRIC,
            "overlap_stages": args.stages,
            "value": value, "unit": "elements/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if partitioned else "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "elements": E, "nodes": N, "ndof": ndof, "nnz": nnz,
                       "scatter": ("chunked fixed point" if (d["form"] == 2 and args.scatter != 1) else "local rows"),
                       "order": d["order"], "form": {0: "poisson", 1: "diffusion+mass", 2: "elasticity"}[d["form"]],
                       "npts": d["npts"], "mesh": f"{d['n']}^3 Kuhn cube, interior nodes perturbed 0.2h",
                       "l2": "256 MB buffer written between timed steps (> 129 MB L2)",
                       "parallelism": (f"row partition x{ws}: each GPU assembles a z-slab of rows with its ghost "
                                       f"elements ({E} of the mesh's {E_total} on rank 0), no communication"
                                       if partitioned else f"independent replica per GPU x{ws}")},
            "roofline": roof,
            "hbm": hbm_block(alg, total_ms / args.steps),
            "fp64_peak_measured_tflops": fp64_peak,
            "fp64_peak_nominal_tflops": FP64_NOMINAL_TFLOPS,
            "forms": forms,
            "pattern_ms": pattern_ms,
            "e2e": e2e,
            "gpu_launches": per_step * args.steps,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out))
    mesh.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0  # fallback copy bandwidth


# ---------------------------------------------------------------- other forms
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# Relative cost of a P2 element against a P1 element in the batch's Poisson
# forms (element kernel + scatter per element of the single-mesh forms: P2
# 64^3 1.26 ms / 1.57M, P1 96^3 1.19 ms / 5.3M), the weight of the batch's
# split over several GPUs.
BATCH_P2_WEIGHT = 3.6


def bench_batched(fea, torch, dev, steps, warmup, flush, ws=1, rank=0):
    """256 uneven meshes (n ~ U{4..32}, half P1 / half P2 Poisson, log-normal
    kappa): one CUDA-graph launch (autotuned) vs one fea_assemble per mesh.
    With several ranks the meshes are split by longest processing time first
    (fea_partition_batch on element counts weighted by order) and each rank
    assembles its own as a batch; the time is the slowest rank's."""
    specs = mg.batch()
    E_all = sum(d["tets"].shape[1] for d in specs)
    if ws > 1:
        sides, orders = mg.batch_sides()
        cost = 6.0 * sides.astype(np.float64) ** 3 * np.where(orders == 2, BATCH_P2_WEIGHT, 1.0)
        part, _ = fea.fea_partition_batch(cost, ws)
        specs = [d for d, p in zip(specs, part) if p == rank]
    meshes, forms, quads, coeffs, keep = [], [], [], [], []
    for d in specs:
        m = fea.Mesh(d["coords"], d["tets"], device=dev)
        kap = torch.as_tensor(d["kappa"], device=dev)
        keep.append(kap)
        meshes.append(m)
        forms.append(fea.make_form(fea.FEA_POISSON, d["order"]))
        quads.append(fea.make_quadrature(d["npts"], fea.FEA_FP64))
        coeffs.append(fea.make_coeffs(kappa=kap, f_kind=fea.FEA_LOAD_SINPROD, f_param=(d["f_amp"],)))
    E = sum(d["tets"].shape[1] for d in specs)
    b = fea.Batch(meshes, forms, quads, coeffs, fea.FEA_LOAD_SINPROD)
    params = b.tune()
    outs = [(b.values[k], b.rhs[k]) for k in range(len(meshes))]

    def graph_step():
        b.assemble()

    def separate_step():
        for m, f, q, c, (v, r) in zip(meshes, forms, quads, coeffs, outs):
            fea.fea_assemble(m.h, f, c, q, v, r)

    res = {}
    for name, fn in (("graph", graph_step), ("separate", separate_step)):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for k in range(steps):
            flush.fill_(k)
            a, c = _events(torch)
            a.record()
            fn()
            c.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(c)
        res[name] = max_over_ranks(tot, dev) / steps
    for m in meshes:
        m.check()
    b.close()
    patterns = [m.pattern(d["order"]) for d, m in zip(specs, meshes)]
    for m in meshes:
        m.close()
    alg = sum(algorithmic_bytes("p1_kappa" if d["order"] == 1 else "p2_diffmass", d["tets"].shape[1],
                                d["coords"].shape[1], nd, nz) for d, (nd, nz) in zip(specs, patterns))
    if ws > 1:
        alg = max_over_ranks(float(alg), dev)  # the largest rank's share
    return {"value": E_all / (res["graph"] / 1e3), "unit": "elements/s", "ms_per_step": res["graph"],
            "hbm": hbm_block(alg, res["graph"]),
            "roofline": None, "roofline_note": "the P1 and P2 element kernels run concurrently in one graph; "
                                                "their FP64 rooflines are those of p1_kappa_96 and p2_diffmass_64",
            "separate_value": E_all / (res["separate"] / 1e3), "separate_ms_per_step": res["separate"],
            "launches": {"graph": 1, "separate": 2 * len(specs)},
            "tuned": {"elements_per_item": params[0], "p2_element_ctas": params[1], "p1_element_ctas": params[2],
                      "scatter_ctas": params[3], "p2_register_variant": params[4], "p1_register_variant": params[5]},
            "meshes": len(specs) if ws == 1 else 256, "elements": E_all,
            "split": (f"{ws} GPUs, meshes by longest processing time first (fea_partition_batch), "
                      f"{len(specs)} meshes / {E} elements on rank {rank}, no communication") if ws > 1 else None,
            "config": "256 Kuhn cubes, n ~ U{4..32} (seed 0), even P1 (4-pt) / odd P2 (11-pt) Poisson, "
                      "log-normal kappa, sin load, FP64"}


def bench_adjoint(fea, torch, dev, steps, warmup, flush, fp64_peak):
    """P1 kappa-diffusion on the 96^3 mesh: forward assembly and the adjoint
    (dL/dkappa, dL/dx for L = v^T K w + g^T f)."""
    d = mg.adjoint_p1(96)
    m = fea.Mesh(d["coords"], d["tets"], device=dev)
    ndof, nnz = m.pattern(1)
    rp, ci = m.pattern_tensors(1)
    rows = torch.repeat_interleave(torch.arange(ndof, device=dev), torch.diff(rp.long()))
    v, w, g = (torch.as_tensor(d[k], device=dev) for k in ("v", "w", "g"))
    gV = v[rows] * w[ci.long()]
    kap = torch.as_tensor(d["kappa"], device=dev)
    form = fea.make_form(fea.FEA_POISSON, 1)
    co = fea.make_coeffs(kappa=kap, f_kind=fea.FEA_LOAD_SINPROD, f_param=(mg.SIN_AMP,))
    q = fea.make_quadrature(4, fea.FEA_FP64)
    E, N = d["tets"].shape[1], d["coords"].shape[1]
    vals = torch.empty(nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(ndof, dtype=torch.float64, device=dev)
    gk = torch.empty(E, dtype=torch.float64, device=dev)
    gx = torch.empty((3, N), dtype=torch.float64, device=dev)
    res = {}
    for name, fn in (("forward", lambda: fea.fea_assemble(m.h, form, co, q, vals, rhs)),
                     ("backward", lambda: fea.fea_assemble_backward(m.h, form, co, q, gV, g, gk, gx))):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for k in range(steps):
            flush.fill_(k)
            a, c = _events(torch)
            a.record()
            fn()
            c.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(c)
        res[name] = tot / steps
    m.check()
    m.close()
    # backward: reads gV (nnz), gF (ndof), coords, tets, kappa; writes
    # dL/dkappa (E) and dL/dx (3 N)
    alg_bwd = 8 * nnz + 8 * ndof + 24 * N + 16 * E + 8 * E + 8 * E + 24 * N
    return {"value": E / (res["backward"] / 1e3), "unit": "elements/s (backward)",
            "backward_ms": res["backward"], "forward_ms": res["forward"],
            "forward_value": E / (res["forward"] / 1e3), "elements": E,
            "roofline": roofline_block("adjoint_96", E, res["backward"], fp64_peak,
                                       note="kernel time taken as the whole backward step (the adjoint kernel "
                                            "and its node reduction)"),
            "hbm": hbm_block(alg_bwd, res["backward"]),
            "config": "P1 kappa-diffusion, 96^3 Kuhn cube (5,308,416 tets), 4-pt sin load, FP64"}


def bench_plain(fea, torch, dev, kind, n, steps, warmup, flush, fp64_peak):
    """FP64 and mixed assembly of one more workload (elements/s each)."""
    d = make_inputs(kind, n, seed=0)
    m = fea.Mesh(d["coords"], d["tets"], device=dev)
    ndof, nnz = m.pattern(d["order"], d["ndpn"])
    keep = []
    if d["form"] == 2:
        lam, mu = torch.as_tensor(d["lam"], device=dev), torch.as_tensor(d["mu"], device=dev)
        keep += [lam, mu]
        co = fea.make_coeffs(lam=lam, mu=mu, f_kind=d["f_kind"], f_param=d["f_param"])
    else:
        kap = None if d["kappa"] is None else torch.as_tensor(d["kappa"], device=dev)
        keep.append(kap)
        co = fea.make_coeffs(kappa=kap, f_kind=d["f_kind"], f_param=d["f_param"])
    form = fea.make_form(d["form"], d["order"], d["mass"])
    vals = torch.empty(nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(ndof, dtype=torch.float64, device=dev)
    fea.fea_profile_enable(m.h, True)
    E = d["tets"].shape[1]
    out = {"elements": E}
    for name, prec in (("fp64", fea.FEA_FP64), ("mixed", fea.FEA_MIXED)):
        q = fea.make_quadrature(d["npts"], prec)
        for _ in range(warmup):
            fea.fea_assemble(m.h, form, co, q, vals, rhs)
        torch.cuda.synchronize()
        tot, pe, ps = 0.0, 0.0, 0.0
        for k in range(steps):
            flush.fill_(k)
            a, c = _events(torch)
            a.record()
            fea.fea_assemble(m.h, form, co, q, vals, rhs)
            c.record()
            e_ms, s_ms = fea.fea_profile_last(m.h)
            tot += a.elapsed_time(c)
            pe += e_ms
            ps += s_ms
        out[name] = {"value": E / (tot / steps / 1e3), "ms_per_step": tot / steps, "elem_ms": pe / steps,
                     "scatter_ms": ps / steps}
        out[name]["hbm"] = hbm_block(algorithmic_bytes(kind, E, d["coords"].shape[1], ndof, nnz), tot / steps)
        if name == "fp64":
            ref = (vals.clone(), rhs.clone())
            key = {"p2_diffmass": "p2_diffmass_64", "p1_kappa": "p1_kappa_96", "p1_poisson": "p1_poisson_8",
                   "elasticity": "p1_elast_128"}[kind]
            note = None
            if n <= 8:
                note = (f"{E} elements, a few microseconds of work: launch-bound, so the fraction says nothing "
                        "about the kernel")
            out[name]["roofline"] = roofline_block(key, E, pe / steps, fp64_peak, note=note)
        else:
            out[name]["error_vs_fp64"] = mixed_error(torch, m, d, ref[0], vals, ref[1], rhs)
    m.check()
    m.close()
    return out


def bench_paper_2d(fea, torch, dev, steps, warmup, flush, fp64_peak, n=2048):
    """The paper's own 2-D example (Sec. 4.2) at the top of its 10K-10M node
    range: P1 triangles on n^2 squares, sigma = [[1, -x-y], [x+y, 1]],
    lambda = 1, f = -2 (x^2 + y^2) + 36, 6-point load rule, FP64."""
    coords, tris = mg.tri_square(n, 0.2, 0)
    m = fea.Mesh(coords, tris, device=dev)
    ndof, nnz = m.pattern(1, 1)
    vals = torch.empty(nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(ndof, dtype=torch.float64, device=dev)
    form = fea.make_form2d()
    fea.fea_profile_enable(m.h, True)
    for _ in range(warmup):
        fea.fea_assemble_2d(m.h, form, vals, rhs)
    torch.cuda.synchronize()
    tot, pe, ps = 0.0, 0.0, 0.0
    for k in range(steps):
        flush.fill_(k)
        a, c = _events(torch)
        a.record()
        fea.fea_assemble_2d(m.h, form, vals, rhs)
        c.record()
        e_ms, s_ms = fea.fea_profile_last(m.h)
        tot += a.elapsed_time(c)
        pe += e_ms
        ps += s_ms
    m.check()
    m.close()
    E = tris.shape[1]
    ms = tot / steps
    alg = 16 * ndof + 12 * E + 8 * nnz + 8 * ndof  # coords, connectivity, values, rhs
    return {"value": E / (ms / 1e3), "unit": "elements/s", "ms_per_step": ms, "elem_ms": pe / steps,
            "scatter_ms": ps / steps, "elements": E, "nodes": ndof, "nnz": nnz,
            "hbm": hbm_block(alg, ms), "roofline": roofline_block("paper_2d", E, pe / steps, fp64_peak),
            "config": f"paper's 2-D example on {n}^2 squares (P1 triangles, perturbed), FP64"}


def bench_jit(fea, torch, dev, steps, warmup, flush, n=64):
    """Runtime-specialised (NVRTC) P2 diffusion + mass on the 64^3 cube:
    compile time, the first call including compile + load, and steady
    throughput - once for the same mathematics as the precompiled headline
    kernel (no k, f = 3 pi^2 sin sin sin) and once with a spatially varying
    coefficient k(x) = 1 + sin(3x) cos(2y) / 2 + z^2 inside the integral."""
    d = make_inputs("p2_diffmass", n, seed=0)
    m = fea.Mesh(d["coords"], d["tets"], device=dev)
    ndof, nnz = m.pattern(2, 1)
    kap = torch.as_tensor(d["kappa"], device=dev)
    co = fea.make_coeffs(kappa=kap, f_param=(mg.SIN_AMP, 0.0, 0.0, 0.0))
    form = fea.make_form(fea.FEA_DIFFUSION_MASS, 2, 1.0)
    q = fea.make_quadrature(11, fea.FEA_FP64)
    vals = torch.empty(nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(ndof, dtype=torch.float64, device=dev)
    fexpr = "p0*sinpi_fx(x)*sinpi_fx(y)*sinpi_fx(z)"
    E = d["tets"].shape[1]
    fea.fea_profile_enable(m.h, True)
    out = {}
    for name, kexpr in (("same_as_headline", None), ("k_of_x", "1 + 0.5*sin(3*x)*cos(2*y) + z*z")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        j = fea.fea_jit_compile(form, q, kexpr, fexpr)
        fea.fea_jit_assemble(m.h, j, co, vals, rhs)
        torch.cuda.synchronize()
        first_ms = (time.perf_counter() - t0) * 1e3
        compile_ms, cubin, hit = fea.fea_jit_info(j)
        for _ in range(warmup):
            fea.fea_jit_assemble(m.h, j, co, vals, rhs)
        torch.cuda.synchronize()
        tot, pe = 0.0, 0.0
        for k in range(steps):
            flush.fill_(k)
            a, c = _events(torch)
            a.record()
            fea.fea_jit_assemble(m.h, j, co, vals, rhs)
            c.record()
            pe += fea.fea_profile_last(m.h)[0]
            tot += a.elapsed_time(c)
        ms = tot / steps
        out[name] = {"value": E / (ms / 1e3), "unit": "elements/s", "ms_per_step": ms, "elem_ms": pe / steps,
                     "compile_ms": compile_ms, "cache_hit": hit, "cubin_bytes": cubin,
                     "first_call_ms_including_compile": first_ms, "k_expr": kexpr, "f_expr": fexpr}
        fea.fea_jit_destroy(j)
    m.check()
    m.close()
    out["config"] = f"P2 diffusion + mass, {n}^3 cube, 11-point rule, FP64, kernels compiled at run time (NVRTC)"
    return out


def bench_solve(fea, torch, dev, n=64, rtol=1e-8, max_iter=3000):
    """The step after assembly on the headline system (P2 diffusion + mass,
    64^3, log-normal kappa): Dirichlet u = 0 on the cube boundary, then
    Jacobi-preconditioned CG to ||r|| <= rtol ||b||.  One solve, timed with
    CUDA events; bytes per iteration = 12 nnz (values, columns) + 108 ndof
    (row pointers and the vectors the five kernels read and write)."""
    d = make_inputs("p2_diffmass", n, seed=0)
    m = fea.Mesh(d["coords"], d["tets"], device=dev)
    ndof, nnz = m.pattern(2, 1)
    kap = torch.as_tensor(d["kappa"], device=dev)
    co = fea.make_coeffs(kappa=kap, f_kind=fea.FEA_LOAD_SINPROD, f_param=(mg.SIN_AMP,))
    form = fea.make_form(fea.FEA_DIFFUSION_MASS, 2, 1.0)
    q = fea.make_quadrature(11)
    ed = m.dof_table(2).cpu().numpy()
    bd, _ = mg.cube_boundary_dofs(d["coords"], ed, ndof)
    bdt = torch.as_tensor(bd, device=dev)
    vals = torch.empty(nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(ndof, dtype=torch.float64, device=dev)
    x = torch.zeros(ndof, dtype=torch.float64, device=dev)
    fea.fea_assemble(m.h, form, co, q, vals, rhs)
    fea.fea_dirichlet(m.h, 2, 1, bdt, None, vals, rhs)
    fea.fea_cg(m.h, 2, 1, vals, rhs, x, rtol=rtol, max_iter=20)  # warm-up: scratch, graph path
    torch.cuda.synchronize()
    a, b, c, e = (torch.cuda.Event(enable_timing=True) for _ in range(4))
    a.record()
    fea.fea_assemble(m.h, form, co, q, vals, rhs)
    b.record()
    fea.fea_dirichlet(m.h, 2, 1, bdt, None, vals, rhs)
    c.record()
    x.zero_()
    it, rel = fea.fea_cg(m.h, 2, 1, vals, rhs, x, rtol=rtol, max_iter=max_iter)
    e.record()
    torch.cuda.synchronize()
    m.check()
    m.close()
    cg_ms = c.elapsed_time(e)
    per_it = cg_ms / max(it, 1)
    bytes_it = 12 * nnz + 108 * ndof
    return {"unit": "ms", "assemble_ms": a.elapsed_time(b), "dirichlet_ms": b.elapsed_time(c), "cg_ms": cg_ms,
            "iterations": it, "rel_residual": rel, "ms_per_iteration": per_it,
            "gbs_per_iteration": bytes_it / (per_it / 1e3) / 1e9,
            "config": f"P2 diffusion + mass {n}^3 (ndof {ndof}, nnz {nnz}), u = 0 on the boundary, Jacobi PCG to "
                      f"rtol {rtol}"}


# ---------------------------------------------------------------- CPU oracle
# Bounded samples of each workload (same recipe, smaller cube) for the CPU
# baseline: each takes some 10-20 s of host time for three repetitions of the
# pattern, the single-threaded values and the all-cores values.
CPU_SAMPLE_N = {"p2_diffmass": 48, "p1_poisson": 64, "p1_kappa": 64, "elasticity": 48}


def _oracle_kw(d):
    return dict(f_kind={1: "const", 2: "sinprod"}[d["f_kind"]], f_param=d["f_param"], npts=d["npts"])


def _oracle_assemble(d, edof, rp, ci):
    import oracle
    kw = _oracle_kw(d)
    if d["form"] == 2:
        return oracle.assemble(d["coords"], d["tets"], 1, edof, rp, ci, kind="elasticity", lam=d["lam"],
                               mu=d["mu"], **kw)
    return oracle.assemble(d["coords"], d["tets"], d["order"], edof, rp, ci, mass=d["mass"], kappa=d["kappa"], **kw)


def _oracle_assemble_par(d, edof, rp, ci):
    import oracle
    kw = _oracle_kw(d)
    if d["form"] == 2:
        return oracle.assemble_par(d["coords"], d["tets"], 1, edof, rp, ci, kind="elasticity", lam=d["lam"],
                                   mu=d["mu"], **kw)
    return oracle.assemble_par(d["coords"], d["tets"], d["order"], edof, rp, ci, mass=d["mass"],
                               kappa=d["kappa"], **kw)


def host_info():
    """Core count and CPU model of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    import platform
    return {"host_cores": os.cpu_count(), "host_cpu": model, "host_arch": platform.machine()}


def cpu_baseline(kind):
    """The oracle, as it stands, on a bounded sample of the workload, on the
    host: the pattern (sort + unique) and the values + load assembly timed
    separately on one thread (median of 3), and the same element loop on all
    host cores (OpenMP, per-thread copies of the outputs summed; median of 3)."""
    import oracle
    n = CPU_SAMPLE_N[kind]
    d = make_inputs(kind, n, seed=0)
    edof, nsd = oracle.dof_table(d["order"], d["coords"].shape[1], d["tets"])
    pat, vals, par = [], [], []
    threads = 1
    for _ in range(3):
        t = time.perf_counter()
        rp, ci = oracle.pattern(nsd, edof, ndpn=d["ndpn"])
        pat.append(time.perf_counter() - t)
    for _ in range(3):
        t = time.perf_counter()
        _oracle_assemble(d, edof, rp, ci)
        vals.append(time.perf_counter() - t)
    for _ in range(3):
        t = time.perf_counter()
        threads = _oracle_assemble_par(d, edof, rp, ci)[3]
        par.append(time.perf_counter() - t)
    E = d["tets"].shape[1]
    pv, vv, av = statistics.median(pat), statistics.median(vals), statistics.median(par)
    out = {"value": E / vv, "unit": "elements/s", "cores": 1, "kind": "oracle",
           "sample": f"{kind} on the {n}^3 cube ({E} tets, {rp[-1]} nonzeros) of the same recipe; value = values + "
                     "load assembly on one thread, pattern timed separately",
           "seconds": vv, "pattern_s": pv, "values_s": vv,
           "all_cores": {"value": E / av, "unit": "elements/s", "cores": threads, "values_s": av,
                         "kind": "the oracle's element loop on OpenMP threads (per-thread copies of the outputs, "
                                 "summed); a timing baseline, not the checker"}}
    out.update(host_info())
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    wl = WORKLOADS[args.workload]
    n = {"p2_diffmass": 32, "p1_poisson": 48, "p1_kappa": 48, "elasticity": 32}[wl["kind"]]
    d = make_inputs(wl["kind"], n, seed=0)
    edof, nsd = oracle.dof_table(d["order"], d["coords"].shape[1], d["tets"])
    rp, ci = oracle.pattern(nsd, edof, ndpn=d["ndpn"])
    E = d["tets"].shape[1]
    for _ in range(args.warmup):
        _oracle_assemble(d, edof, rp, ci)
    t = time.perf_counter()
    for _ in range(args.steps):
        _oracle_assemble(d, edof, rp, ci)
    dt = time.perf_counter() - t
    value = E * args.steps / dt
    out = {
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "elements/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample_elements": E,
                   "note": f"each step assembles a {n}^3 cube of the same recipe (bounded CPU sample)"},
        "cpu_baseline": dict({"value": value, "unit": "elements/s", "cores": 1, "kind": "oracle",
                              "sample": f"{wl['kind']} on the {n}^3 cube ({E} tets) per step"}, **host_info()),
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="p1_elast_128", choices=sorted(WORKLOADS))
    p.add_argument("--scatter", type=int, default=0, help="0 automatic, 1 local rows, 2 chunked (elasticity)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--replicas", action="store_true",
                   help="with several GPUs, every rank assembles its own copy of the workload (weak scaling) "
                        "instead of a row partition of one mesh")
    p.add_argument("--stages", type=int, default=1, help="element chunks overlapped with the scatter (1 = none)")
    p.add_argument("--scatter-classes", type=int, default=-1, help="scatter launch shape 0-3 (-1 = library default)")
    p.add_argument("--scatter-stages", type=int, default=0,
                   help="bulk-copy scatter stages per CTA, 2-4 (0 = library default)")
    p.add_argument("--load-split", type=int, default=-1, help="element launch: 0 fused, 1 matrix then load, "
                                                               "2 load kernel concurrent with the matrix kernel "
                                                               "(-1 = library default)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-forms", action="store_true")
    p.add_argument("--forms", default="all",
                   help="comma list of extra forms to time: mixed, local_rows, atomic_alg1, batched, adjoint, "
                        "p2_diffmass_64, elasticity_128, p1_kappa_96, p1_poisson_8, paper_2d, jit, solve "
                        "(default all)")
    args = p.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
