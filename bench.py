"""Benchmark: element matrices/s and assembled nnz/s of the P3 stiffness +
mass workload on tetrahedra (unit cube, 24^3 boxes x 6 Kuhn tetrahedra =
82,944 cells, vertices jittered +-0.15h, kappa lognormal(0,1) at the 64
points of the 6-exact collapsed Gauss-Jacobi rule), mixed precision (BF16
operands, FP32 accumulation) against the FP64 GPU path.

One step = element matrices of both forms (written to HBM) + their CSR
assembly, through the C ABI (fe_assemble).  Inputs are resident in HBM; the
L2 is flushed between timed steps: a 512 MB write, then a read of the same
buffer so that the write-back of the evicted dirty lines also happens outside
the timed events (L2 then holds only clean lines of the flush buffer).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank runs an independent copy of the workload (weak
scaling, no collective); rank 0 prints the JSON line with the max-over-ranks
time.  --impl reference times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores (rank 0 only).
"""
from __future__ import annotations

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

WORKLOAD = ("P3 stiffness + mass, unit cube 24^3 boxes x 6 Kuhn tetrahedra (82,944 cells, 389,017 dofs, "
            "18,388,729 nnz per matrix), jitter +-0.15h, kappa lognormal(0,1) at 64 collapsed Gauss-Jacobi points")
METRIC = "element matrices/s and assembled nnz/s, mixed vs FP64 GPU, at stated max rel error"


def max_over_ranks(x, world, device="cuda"):
    """The largest value of x over all ranks (a job's time is its slowest
    rank's); x itself on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step, ms_per_step, world):
    """Whole-job units per second: every rank processes its own units in the
    (max-over-ranks) step time."""
    return world * units_per_rank_step / (ms_per_step / 1e3)


def workload_config(world):
    """The `config` of both arms: the workload and how steps are timed."""
    return {"workload": WORKLOAD,
            "step": "element matrices of both forms (stiffness + mass) + CSR assembly of both",
            "l2": "flushed between steps (512 MB write, then a read of it, outside the timed events)",
            "parallelism": f"independent replica per GPU x{world}"}
N_BOX, DEGREE, ALPHA, SEED_MESH, SEED_KAPPA = 24, 3, 0.15, 2, 3


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.samples = []
        self.proc = None
        self.index = index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for n, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def make_inputs():
    from paper_2410_12614_gb300 import inputs
    v, c = inputs.cube_mesh(N_BOX, ALPHA, SEED_MESH)
    return v, c


def algorithmic_bytes(plan, prec):
    """Bytes each kernel must move through HBM per launch (both forms).

    factor:   kappa (FP64) + connectivity + vertices in; FP32 window (n_q padded
              to 4) + 64-byte per-cell factor record out.
    element:  window + the 48 used bytes of the factor record in; element
              matrices of both forms out (the shared operand P stays in L2).
    assembly: element matrices of both forms, a 2-byte stage position per
              element entry, a 1-byte segment length per CSR value and the
              incidence list in; CSR values of both forms out.
    """
    eb = 8 if prec == "fp64" else 4
    nc, nph, nq = plan.n_cells, plan.n_phi, plan.n_q
    ldw = (nq + 3) // 4 * 4
    d = plan.d
    factor = nc * nq * 8 + nc * (d + 1) * 4 + plan.n_vertices * d * 8 + nc * ldw * 4 + nc * 64
    elem = nc * ldw * 4 + nc * 48 + 2 * nc * nph * nph * eb
    asm = 2 * nc * nph * nph * eb + nc * nph * nph * 2 + plan.nnz + nc * nph * 4 + 2 * plan.nnz * eb
    return factor, elem, asm


def action_cost(plan):
    """Algorithmic HBM bytes and FP32 flops of one action step (both forms in
    one pass): kappa (FP64), connectivity, vertices and the cells' dof lists in
    once; each global coefficient read once (later gathers hit L2); per form,
    the cell vectors written and read back by the vector assembly, and the
    assembled vector out; the incidence lists read once.  Flops: grad w (or w)
    at the points, r, and b."""
    nc, nq, nph, d, nd_ = plan.n_cells, plan.n_q, plan.n_phi, plan.d, plan.n_dofs
    shared = (8 * nq * nc + 4 * (d + 1) * nc + 8 * d * plan.n_vertices + 4 * nph * nc + 8 * nd_
              + 8 * (nd_ + 1) + 4 * nph * nc)
    per_form = 2 * 4 * nph * nc + 4 * nd_
    flops = nc * nq * (2 * d * nph + (2 * d * d + d) + 2 * d * nph)   # Poisson
    flops += nc * nq * (2 * nph + 2 + 2 * nph)                         # mass
    return shared + 2 * per_form, flops


def _traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/traffic.json), if the kernel's sources are unchanged since the
    capture (else None)."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, "paper_2410_12614_gb300", "csrc", f), "rb").read())
        if h.hexdigest() != rec["sha256"]:
            return None
        return rec["dram_bytes_per_launch"]
    except (OSError, KeyError, ValueError):
        return None


_FP64_PEAK = None


def measured_fp64_peak():
    """FP64 peak of this GPU measured as a cuBLAS DGEMM burst (torch.matmul on
    float64, 6144^3, best of 3, CUDA events), measured once per process."""
    global _FP64_PEAK
    if _FP64_PEAK is not None:
        return _FP64_PEAK
    import torch
    n = 6144
    a = torch.randn((n, n), dtype=torch.float64, device="cuda")
    b = torch.randn((n, n), dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 1e30
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    _FP64_PEAK = 2.0 * n ** 3 / (best / 1e3) / 1e12
    return _FP64_PEAK


def fp64_peak_and_fraction(plan, element_ms):
    peak = measured_fp64_peak()
    nph, nq = plan.n_phi, plan.n_q
    nsym = nph * (nph + 1) // 2
    flops = 0
    for nd in (3, 1):
        flops += 2 * nd * nq * nsym + 2 * nd * nd * nq * nph
    flops *= plan.n_cells
    got = flops / (element_ms / 1e3) / 1e12
    return {"fp64_peak_tflops": peak, "fp64_peak_source": "measured: torch.matmul float64 6144^3 (cuBLAS DGEMM), "
                                                          "best of 3, CUDA events",
            "element_kernel_fp64_flops": flops, "element_kernel_fp64_tflops": got, "frac_of_fp64_peak": got / peak}


def run_ours(args, rank, world):
    import torch
    from paper_2410_12614_gb300 import api, inputs

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    v, c = make_inputs()
    pts, w = api.quadrature_rule("tetrahedron", DEGREE + 1)
    with torch.cuda.stream(stream):
        plan = api.Plan("tetrahedron", v, c, DEGREE, pts, w, precisions=("bf16", "fp16"), stream=stream)
        kap_h = inputs.lognormal_kappa(plan.n_cells, plan.n_q, SEED_KAPPA)
        kap = torch.from_numpy(kap_h).cuda()
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        flush_sink = torch.empty((), dtype=torch.float32, device="cuda")

        def buffers(prec):
            els = {f: plan.empty_elements(prec) for f in ("stiffness", "mass")}
            vals = {f: plan.empty_values(prec) for f in ("stiffness", "mass")}
            return els, vals

        def timed(prec, steps, warmup):
            """Step times with the library's stage events off (the events would add
            their own latency), then per-kernel stage times from a second pass of
            the same steps with the events on."""
            els, vals = buffers(prec)
            plan.enable_timing(False)
            for _ in range(warmup):
                plan.assemble(kap, prec=prec, elements=els, out=vals)
            plan.sync()
            step_ms = []
            launches = 0
            for _ in range(steps):
                flush.fill_(1.0)
                flush_sink.copy_(flush.sum())   # reads the 512 MB back: dirty lines written back here
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plan.assemble(kap, prec=prec, elements=els, out=vals)
                e1.record(stream)
                launches += plan.last_launches()
                stream.synchronize()
                step_ms.append(e0.elapsed_time(e1))
            plan.sync()
            el_ms, as_ms, fa_ms = [], [], []
            plan.enable_timing(True)
            for _ in range(max(3, steps // 2)):
                flush.fill_(1.0)
                flush_sink.copy_(flush.sum())
                plan.assemble(kap, prec=prec, elements=els, out=vals)
                stream.synchronize()
                st = plan.stage_times()
                el_ms.append(st[0])
                as_ms.append(st[1])
                fa_ms.append(st[3])
            plan.sync()
            plan.enable_timing(False)
            return step_ms, (fa_ms, el_ms, as_ms), launches, els, vals

        # headline: BF16
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(dev)
        sampler.start()
        step_ms, (fa_ms, el_ms, as_ms), launches, els, vals = timed("bf16", args.steps, args.warmup)
        clocks = sampler.stop()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        total_ms = max_over_ranks(sum(step_ms), world)
        ms_step = total_ms / args.steps
        elems_per_step = 2 * plan.n_cells
        value = job_throughput(elems_per_step, ms_step, world)
        nnz_per_s = job_throughput(2 * plan.nnz, ms_step, world)

        # end to end through the public API with host buffers: a sequence of
        # `steps` coefficient sets through fe_assemble_host_many (each item's
        # kappa uploaded from pinned host memory and its CSR values downloaded,
        # uploads, compute and downloads overlapped), and single
        # fe_assemble_host calls for comparison
        kap_pinned = torch.from_numpy(kap_h).pin_memory()
        host_out = [{f: torch.empty(plan.nnz, dtype=torch.float32, pin_memory=True) for f in ("stiffness", "mass")}
                    for _ in range(2)]
        seq_k = [kap_pinned] * args.steps
        seq_o = [host_out[i % 2] for i in range(args.steps)]
        plan.assemble_host_many(seq_k[:4], seq_o[:4], prec="bf16")
        e2e_runs = []
        for _ in range(3):
            t0 = time.perf_counter()
            plan.assemble_host_many(seq_k, seq_o, prec="bf16")
            e2e_runs.append((time.perf_counter() - t0) * 1e3 / args.steps)
        e2e_step = max_over_ranks(statistics.median(e2e_runs), world)
        for _ in range(2):
            plan.assemble_host(kap_pinned, prec="bf16", out=host_out[0])
        single_ms = []
        for _ in range(max(3, args.steps // 2)):
            t0 = time.perf_counter()
            plan.assemble_host(kap_pinned, prec="bf16", out=host_out[0])
            single_ms.append((time.perf_counter() - t0) * 1e3)
        single_step = max_over_ranks(statistics.median(single_ms), world)

        # other precisions (context lines)
        extra = {}
        for prec, k in (("fp16", max(3, args.steps // 2)), ("fp64", 3)):
            s2, (f2, e2, a2), _, _, _ = timed(prec, k, 1)
            extra[prec] = {"ms_per_step": statistics.mean(s2), "factor_kernel_ms": statistics.mean(f2),
                           "element_kernel_ms": statistics.mean(e2), "assembly_kernel_ms": statistics.mean(a2),
                           "element_matrices_per_s": elems_per_step / (statistics.mean(s2) / 1e3)}
        extra["bf16_speedup_vs_fp64"] = extra["fp64"]["ms_per_step"] / ms_step
        # the FP64 comparator against a measured FP64 peak: a cuBLAS DGEMM burst
        # (torch.matmul on float64, 6144^3, best of 3, CUDA events), the same
        # method as the BF16 peak of MEASURED_PEAKS.json; the FP64 element kernel's
        # flops are those of its H~-form with symmetry per cell and form:
        # 2 n_d n_q n_sym + 2 n_d^2 n_q n_phi
        extra["fp64"].update(fp64_peak_and_fraction(plan, extra["fp64"]["element_kernel_ms"]))

        # linear forms (Algorithm 2): both forms' actions on a FE function and their vector assembly
        w_d = torch.from_numpy(inputs.gaussian_vector(plan.n_dofs, 9).astype(np.float64)).cuda()
        action = {}
        for prec in ("bf16", "fp64"):
            vbuf = {f: torch.empty(plan.n_dofs, dtype=torch.float64 if prec == "fp64" else torch.float32,
                                   device="cuda") for f in ("stiffness", "mass")}
            for _ in range(3):
                plan.action(kap, w_d, prec=prec, out=vbuf)
            plan.sync()
            ts = []
            for _ in range(max(3, args.steps // 2)):
                flush.fill_(1.0)
                flush_sink.copy_(flush.sum())
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plan.action(kap, w_d, prec=prec, out=vbuf)
                e1.record(stream)
                stream.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            action[prec] = {"ms_per_step": ms, "cell_vectors_per_s": 2 * plan.n_cells / (ms / 1e3)}
        # the mixed action's roofline: max(bytes / HBM peak, flops / FP32 CUDA-core peak), the
        # latter from the unit counts: SMs x 128 FP32 lanes x 2 flops x the maximum SM clock
        hbm_peak, _ = _peaks()
        a_bytes, a_flops = action_cost(plan)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        fp32_tflops = sms * 128 * 2 * (clocks.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
        t_bytes = a_bytes / (hbm_peak * 1e9) * 1e3
        t_flops = a_flops / (fp32_tflops * 1e12) * 1e3
        action["bf16"].update({
            "algorithmic_bytes": a_bytes, "fp32_flops": a_flops,
            "achieved_gbs": a_bytes / (action["bf16"]["ms_per_step"] / 1e3) / 1e9,
            "achieved_fp32_tflops": a_flops / (action["bf16"]["ms_per_step"] / 1e3) / 1e12,
            "fp32_peak_tflops": fp32_tflops, "hbm_peak_gbs": hbm_peak,
            "bound": "alu" if t_flops > t_bytes else "hbm",
            "roofline_ms": max(t_bytes, t_flops),
            "frac_of_roofline": max(t_bytes, t_flops) / action["bf16"]["ms_per_step"]})
        extra["action_algorithm2"] = action

    hbm, how = _peaks()
    fb, eb, ab = algorithmic_bytes(plan, "bf16")
    fa_avg, el_avg, as_avg = statistics.mean(fa_ms), statistics.mean(el_ms), statistics.mean(as_ms)
    kernels = {"factor_kernel": ("factor (geometry + coefficient window)", fa_avg, fb),
               "tc_element_kernel": ("element matrices (tcgen05 BF16)", el_avg, eb),
               "assemble_kernel": ("assembly (chunked segmented reduction)", as_avg, ab)}
    dom_key = max(kernels, key=lambda k: kernels[k][1])
    dom, dom_ms, dom_bytes = kernels[dom_key]
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    result = {
        "metric": METRIC,
        "value": value,
        "unit": "element matrices/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16",
        "data": "synthetic (seeded structured mesh + lognormal kappa)",
        "config": workload_config(world),
        "method": "fe_assemble, BF16 operands on the tcgen05 tensor cores, FP32 accumulation, FP64 geometry; "
                  "element matrices of both forms to HBM, then the CSR values of both",
        "nnz_per_s": nnz_per_s,
        "stage_ms": {"factor_kernel": fa_avg, "element_kernel": el_avg, "assembly_kernel": as_avg,
                     "how": "a second pass of the same steps with the library's stage events on "
                            "(the headline steps run without them)"},
        "kernels": {k: {"ms": v[1], "algorithmic_bytes": v[2], "achieved_gbs": v[2] / (v[1] / 1e3) / 1e9,
                        "frac_of_peak": v[2] / (v[1] / 1e3) / 1e9 / hbm, "traffic": _traffic(k)}
                    for k, v in kernels.items()},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": _traffic(dom_key),
                     "peak_source": f"{how} (MEASURED_PEAKS.json hbm_gbs, copy burst)",
                     "algorithmic_bytes_per_launch": dom_bytes},
        "e2e": {"value": job_throughput(elems_per_step, e2e_step, world), "unit": "element matrices/s",
                "h2d_bytes_per_step": int(plan.n_cells * plan.n_q * 8),
                "d2h_bytes_per_step": int(2 * plan.nnz * 4), "ms_per_step": e2e_step,
                "api": f"fe_assemble_host_many over {args.steps} coefficient sets (pinned host kappa in, pinned "
                       "host CSR values out per item; uploads, compute and downloads overlapped), wall time / items, "
                       "median of 3 sequences",
                "single_call_ms_per_step": single_step,
                "single_call_api": "fe_assemble_host (one synchronous call: upload, compute, download in turn)"},
        "gpu_launches": launches,
        "clocks": clocks,
        "per_precision": extra,
    }
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args, plan, kap_h, els, v, c)
    if rank == 0 and args.with_batch:
        result["batched_256_meshes"] = run_batch(args)
    if rank == 0 and args.sweep:
        result["degree_sweep"] = run_sweep(args)
    if rank == 0 and args.configs:
        result["small_configs"] = run_configs(args)
    if rank == 0 and args.boxed_sweep:
        result["boxed_sweep"] = run_boxed_sweep(args)
    if rank == 0 and not args.headline_only:
        # compact context lines of the other configurations, recorded with every run:
        # the high-degree tetrahedra (P5, P7), Q3 hexahedra against FP64, and the
        # small configurations (P1 Laplace latency, P2 adjoints, fused assembly)
        sargs = argparse.Namespace(**vars(args))
        sargs.sweep_degrees, sargs.sweep_precisions = "5,7", "bf16,e4m3,fp64"
        result["context"] = {"degree_sweep_tet16": run_sweep(sargs),
                             "boxed_q3_hex16": run_boxed_sweep(args, degrees=[3], precs=("bf16", "e4m3")),
                             "small_configs": result.get("small_configs") or run_configs(args)}
    return result


def run_configs(args):
    """The two small configurations beside the headline:
    P1 Laplace in FP64 on 32^2 x 2 triangles (2,048 cells, jitter 0.2h, seed 1,
    kappa = 1, the 3-point rule): element matrices + CSR, a launch-latency-bound
    case reported in microseconds per call (eager) and per CUDA-graph replay;
    the adjoint of the P2 stiffness form on 32^3 x 6 tetrahedra (196,608 cells,
    kappa lognormal at 27 points, u, v ~ N(0,1) FP32): dL/dkappa, dL/dx and L
    by fe_adjoint, and the same for a general gradient on the CSR values by
    fe_adjoint_values, each against its HBM bytes (L2 flushed before each run)."""
    import torch
    from paper_2410_12614_gb300 import api, inputs
    hbm, _ = _peaks()
    out = {}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        v, c = inputs.square_mesh(32, 0.2, 1)
        pts, w = api.quadrature_rule("triangle", 0, family=api._lib.FE_QUAD_TRIANGLE_3POINT)
        plan = api.Plan("triangle", v, c, 1, pts, w, forms=("stiffness",), precisions=("bf16",), stream=stream)
        kap = torch.ones((plan.n_cells, plan.n_q), dtype=torch.float64, device="cuda")
        els = {"stiffness": plan.empty_elements("fp64")}
        vals = {"stiffness": plan.empty_values("fp64")}

        def call():
            plan.assemble(kap, forms=("stiffness",), prec="fp64", elements=els, out=vals)

        for _ in range(5):
            call()
        plan.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 200
        e0.record(stream)
        for _ in range(n):
            call()
        e1.record(stream)
        stream.synchronize()
        c1 = {"workload": "P1 Laplace FP64, 32^2 x 2 triangles (2,048 cells, 1,089 dofs, 7,361 nnz), kappa = 1",
              "us_per_call": e0.elapsed_time(e1) * 1e3 / n, "launches_per_call": plan.last_launches(),
              "note": "back-to-back calls on one stream, inputs L2-resident: launch-latency bound"}
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for _ in range(10):
                    call()
            g.replay()
            stream.synchronize()
            e0.record(stream)
            for _ in range(20):
                g.replay()
            e1.record(stream)
            stream.synchronize()
            c1["us_per_call_graph"] = e0.elapsed_time(e1) * 1e3 / (20 * 10)
        except Exception as ex:   # capture is reported, not required
            c1["us_per_call_graph"] = None
            c1["graph_error"] = str(ex)[:200]
        out["p1_laplace_fp64"] = c1
        del plan

        v, c = inputs.cube_mesh(32, 0.15, 7)
        pts, w = api.quadrature_rule("tetrahedron", 3)
        plan = api.Plan("tetrahedron", v, c, 2, pts, w, forms=("stiffness",), precisions=("bf16",), stream=stream)
        kap = torch.from_numpy(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 7)).cuda()
        u = torch.from_numpy(inputs.gaussian_vector(plan.n_dofs, 8)).cuda()
        vv = torch.from_numpy(inputs.gaussian_vector(plan.n_dofs, 9)).cuda()
        gvals = torch.from_numpy(inputs.gaussian_vector(plan.nnz, 10).astype(np.float64)).cuda()
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        nc, nq, nph, nv = plan.n_cells, plan.n_q, plan.n_phi, plan.n_vertices
        d = 3
        base = (8 * nq * nc * 2 + 16 * nc + 24 * nv + 4 * nph * nc + 96 * nc * 2 + 16 * nc + 8 * (nv + 1)
                + 24 * nv + 16 * nc)
        # FP64 flops per cell and point: the reference gradients (or the block
        # contraction), their products with K, the kappa gradient and S
        fl_uv = nc * nq * (4 * nph * d + 6 * d * d + 2 * d)
        fl_val = nc * nq * (2 * nph * nph * d + 2 * nph * d * d + 4 * d * d)
        for name, fn, nbytes, flops in (
                ("adjoint_quadratic_form", lambda: plan.adjoint(kap, u, vv), base + 8 * plan.n_dofs, fl_uv),
                ("adjoint_values", lambda: plan.adjoint_values(kap, gvals), base + 8 * plan.nnz, fl_val)):
            for _ in range(2):
                fn()
            plan.sync()
            ts = []
            for _ in range(7):
                flush.fill_(1.0)
                flush.sum()
                e0.record(stream)
                fn()
                e1.record(stream)
                stream.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            out[name] = {"workload": "P2 stiffness adjoint, 32^3 x 6 tetrahedra (196,608 cells), FP64",
                         "ms": ms, "cells_per_s": nc / (ms / 1e3), "algorithmic_bytes": nbytes,
                         "achieved_gbs": nbytes / (ms / 1e3) / 1e9, "frac_of_hbm": nbytes / (ms / 1e3) / 1e9 / hbm,
                         "fp64_flops": flops, "achieved_fp64_tflops": flops / (ms / 1e3) / 1e12,
                         "bound": "alu", "fp64_peak_tflops": measured_fp64_peak(),
                         "fp64_peak_source": "measured cuBLAS DGEMM burst",
                         "frac_of_fp64_peak": flops / (ms / 1e3) / 1e12 / measured_fp64_peak()}
        del plan

        # the fused assembly (no element matrices written out) against the unfused
        # one on the same mesh: P2 stiffness + mass, BF16, CSR of both forms
        plan = api.Plan("tetrahedron", v, c, 2, pts, w, precisions=("bf16",), stream=stream)
        kap = torch.from_numpy(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 7)).cuda()
        vals = {f: plan.empty_values("bf16") for f in ("stiffness", "mass")}
        els = {f: plan.empty_elements("bf16") for f in ("stiffness", "mass")}
        res = {"workload": "P2 stiffness + mass, 32^3 x 6 tetrahedra (196,608 cells, 274,625 dofs, 7,678,721 nnz "
                           "per matrix), BF16, CSR of both forms",
               "fused_active": plan.set_fusion(1)}
        for name, fn in (("fused", lambda: plan.assemble(kap, prec="bf16", out=vals)),
                         ("unfused", lambda: plan.assemble(kap, prec="bf16", elements=els, out=vals))):
            for _ in range(3):
                fn()
            plan.sync()
            ts = []
            for _ in range(9):
                flush.fill_(1.0)
                flush.sum()
                e0.record(stream)
                fn()
                e1.record(stream)
                stream.synchronize()
                ts.append(e0.elapsed_time(e1))
            res[name + "_ms"] = statistics.median(ts)
            res[name + "_launches"] = plan.last_launches()
        res["element_matrices_per_s_fused"] = 2 * plan.n_cells / (res["fused_ms"] / 1e3)
        res["speedup_fused_vs_unfused"] = res["unfused_ms"] / res["fused_ms"]
        out["p2_assembly_fused"] = res
    return out


SWEEP_PRECISIONS = ("bf16", "fp16", "tf32", "tf32x3", "e4m3")


def run_sweep(args):
    """Degree sweep: P1..P8 tetrahedra on 16^3 x 6 Kuhn boxes (24,576 cells,
    jitter 0.15h, seed 4; kappa lognormal at (p+1)^3 points, seed 5), element
    matrices of both forms (factor kernel + contraction; FP64 on the CUDA cores
    up to P5) per precision, inputs resident, L2 flushed before each timed run.
    Roofline per run: max(bytes / HBM peak, flops / the format's dense peak)
    with flops = 2 n_d n_q n_phi^2 per cell and form (the Remark after
    Algorithm 1; n_d = 3 Poisson, 1 mass) and bytes = kappa + connectivity
    in, both element matrices out.  Format peaks from the measured BF16 burst
    rate: FP16 the same, TF32 half, E4M3 twice, TF32x3 (three TF32 products
    per term) a sixth."""
    import torch
    from paper_2410_12614_gb300 import api, inputs
    hbm, _ = _peaks()
    try:
        bf16 = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
        peak_src = "measured BF16 burst"
    except Exception:
        bf16, peak_src = 1900.0, "fallback BF16"
    peaks = {"bf16": bf16, "fp16": bf16, "tf32": bf16 / 2, "e4m3": 2 * bf16, "tf32x3": bf16 / 6}
    v, c = inputs.cube_mesh(16, 0.15, 4)
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {"mesh": "P1..P8 tetrahedra, 16^3 boxes x 6 (24,576 cells)", "peaks_tflops": peaks,
           "peak_source": peak_src, "hbm_gbs": hbm, "runs": []}
    degrees = [int(x) for x in args.sweep_degrees.split(",")]
    precs = tuple(x for x in args.sweep_precisions.split(",") if x in SWEEP_PRECISIONS)
    with torch.cuda.stream(stream):
        for p in degrees:
            pts, w = api.quadrature_rule("tetrahedron", p + 1)
            plan = api.Plan("tetrahedron", v, c, p, pts, w, precisions=precs, stream=stream, elements_only=True)
            kap = torch.from_numpy(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 5)).cuda()
            nc, nq, nph = plan.n_cells, plan.n_q, plan.n_phi
            flops = 2.0 * (3 + 1) * nq * nph * nph * nc
            with_fp64 = p <= 5 and "fp64" in args.sweep_precisions.split(",")
            for prec in precs + (("fp64",) if with_fp64 else ()):
                eb = 8 if prec == "fp64" else 4
                els = {f: plan.empty_elements(prec) for f in ("stiffness", "mass")}
                nbytes = nc * (8 * nq + 4 * 4 + 2 * eb * nph * nph) + plan.n_vertices * 3 * 8
                for _ in range(2):
                    plan.element_matrices(kap, prec=prec, out=els)
                plan.sync()
                ts = []
                # the timed launches sit in an NVTX range "timed", so that a profiler
                # can select them (ncu --nvtx --nvtx-include timed/) past the plan's
                # autotuning launches
                torch.cuda.nvtx.range_push("timed")
                for _ in range(5 if prec != "fp64" or p <= 3 else 2):
                    flush.fill_(1.0)
                    flush.sum()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    plan.element_matrices(kap, prec=prec, out=els)
                    e1.record(stream)
                    stream.synchronize()
                    ts.append(e0.elapsed_time(e1))
                torch.cuda.nvtx.range_pop()
                ms = statistics.median(ts)
                run = {"p": p, "prec": prec, "n_phi": nph, "n_q": nq, "ms": ms,
                       "element_matrices_per_s": 2 * nc / (ms / 1e3),
                       "tflops": flops / (ms / 1e3) / 1e12, "gbs": nbytes / (ms / 1e3) / 1e9}
                if prec != "fp64":
                    t_bytes, t_flops = nbytes / (hbm * 1e9), flops / (peaks[prec] * 1e12)
                    run.update({"bound": "tensor" if t_flops > t_bytes else "hbm",
                                "frac_of_roofline": max(t_bytes, t_flops) / (ms / 1e3)})
                out["runs"].append(run)
                del els
            del plan, kap
            torch.cuda.empty_cache()
    return out


def run_boxed_sweep(args, degrees=None, precs=("bf16", "fp16", "e4m3"), n_by_degree=None):
    """Boxed cells (the paper's 60x case is hexahedra): Q_p hexahedra on a
    jittered structured mesh of N^3 cells (N = 34: 39,304 cells, two full waves
    of 128-cell tiles; Q5: N = 32), element-matrix-only plans (no CSR pattern,
    as the paper's kernel experiments), kappa lognormal at the (p+1)^3 tensor
    Gauss-Legendre points, element matrices of both forms per precision and in
    FP64 (per-point FP64 geometry in every path), inputs resident, L2 flushed
    before each timed run; the tensor-core speed-up over the FP64 path and the
    fraction of the roofline as in run_sweep."""
    import torch
    from paper_2410_12614_gb300 import api, inputs
    hbm, _ = _peaks()
    try:
        bf16 = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        bf16 = 1900.0
    peaks = {"bf16": bf16, "fp16": bf16, "tf32": bf16 / 2, "e4m3": 2 * bf16, "tf32x3": bf16 / 6}
    degrees = degrees or [int(x) for x in args.boxed_degrees.split(",")]
    n_by_degree = n_by_degree or {1: 34, 2: 34, 3: 34, 4: 34, 5: 32}
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {"mesh": "Q_p hexahedra, N^3 jittered cells (N = 34, Q5: 32), element-matrix-only plans", "runs": []}
    with torch.cuda.stream(stream):
        for p in degrees:
            n = n_by_degree.get(p, 10)
            v, c = inputs.hex_mesh(n, 0.15, 40 + p)
            plan = api.Plan("hexahedron", v, c, p, precisions=precs, stream=stream, elements_only=True)
            kap = torch.from_numpy(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 50 + p)).cuda()
            nc, nq, nph = plan.n_cells, plan.n_q, plan.n_phi
            flops = 2.0 * (3 + 1) * nq * nph * nph * nc
            times = {}
            for prec in precs + ("fp64",):
                eb = 8 if prec == "fp64" else 4
                els = {f: plan.empty_elements(prec) for f in ("stiffness", "mass")}
                nbytes = nc * (8 * nq + 8 * 4 + 2 * eb * nph * nph) + plan.n_vertices * 3 * 8
                for _ in range(2):
                    plan.element_matrices(kap, prec=prec, out=els)
                plan.sync()
                ts = []
                for _ in range(5 if prec != "fp64" else 3):
                    flush.fill_(1.0)
                    flush.sum()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    plan.element_matrices(kap, prec=prec, out=els)
                    e1.record(stream)
                    stream.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = statistics.median(ts)
                times[prec] = ms
                run = {"p": p, "cells": nc, "prec": prec, "n_phi": nph, "n_q": nq, "ms": ms,
                       "element_matrices_per_s": 2 * nc / (ms / 1e3), "tflops": flops / (ms / 1e3) / 1e12}
                if prec != "fp64":
                    t_bytes, t_flops = nbytes / (hbm * 1e9), flops / (peaks[prec] * 1e12)
                    run.update({"bound": "tensor" if t_flops > t_bytes else "hbm",
                                "frac_of_roofline": max(t_bytes, t_flops) / (ms / 1e3)})
                out["runs"].append(run)
                del els
            for prec in precs:
                out["runs"].append({"p": p, "speedup_vs_fp64": {prec: times["fp64"] / times[prec]}})
            del plan, kap
            torch.cuda.empty_cache()
    return out


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(args, plan=None, kap=None, gpu_els=None, v=None, c=None, budget_s=None):
    """Time the FP64 oracle (single thread, as it stands) on a bounded sample
    of cells of the same workload; with GPU results at hand, also report the
    measured error of the GPU's BF16 element matrices on those cells."""
    import oracle
    from paper_2410_12614_gb300 import inputs

    if v is None:
        v, c = make_inputs()
    pts, w = oracle.collapsed_rule("tetrahedron", DEGREE + 1)
    ref = oracle.Problem(v, c, DEGREE, pts, w)
    if kap is None:
        kap = inputs.lognormal_kappa(ref.n_cells, ref.n_q, SEED_KAPPA)
    budget = budget_s if budget_s is not None else args.cpu_seconds
    # calibrate on 64 cells, then size the sample to the budget
    ids = np.arange(64)
    t0 = time.perf_counter()
    for form in ("stiffness", "mass"):
        ref.element_matrices_subset(kap, form, ids)
    per_cell = (time.perf_counter() - t0) / 64
    n = int(max(128, min(ref.n_cells, budget / max(per_cell, 1e-9))))
    rng = np.random.default_rng(99)
    ids = np.sort(rng.choice(ref.n_cells, size=n, replace=False))
    ref.csr_pattern()  # the pattern is set-up work, outside the timed region
    t0 = time.perf_counter()
    A = {f: ref.element_matrices_subset(kap, f, ids) for f in ("stiffness", "mass")}
    for f in ("stiffness", "mass"):
        ref.assemble_subset(A[f], ids)
    dt = time.perf_counter() - t0
    out = {"value": 2 * n / dt, "unit": "element matrices/s", "cores": 1, "kind": "oracle",
           "sample": f"{n} random cells of the workload: both forms by FP64 literal quadrature loops, "
                     "assembled into the CSR values", "seconds": dt,
           "cpu": _cpu_model()}
    if budget_s is None:
        try:
            out["all_cores"] = cpu_baseline_all_cores(budget, dt / (2 * n) * 2)
        except Exception as e:  # informational only
            out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    if gpu_els is not None:
        import oracle as orc
        errs = {}
        for f in ("stiffness", "mass"):
            got = gpu_els[f][ids].double().cpu().numpy()
            e = np.abs(got - A[f]).reshape(n, -1).max(1) / np.abs(A[f]).reshape(n, -1).max(1)
            kq = ref.kappa_q(kap, f, A[f], cell_ids=ids)
            K = ref.n_q * (6 if f == "stiffness" else 1)
            bnd = orc.error_bound(kq, 2.0 ** -8, K)
            errs[f] = {"max_rel_err": float(e.max()), "max_rel_err_over_u_s": float(e.max() / 2.0 ** -8),
                       "bound_at_worst_cell": float(bnd[np.argmax(e)]), "within_bound": bool(np.all(e <= bnd))}
        out["bf16_accuracy_on_sample"] = errs
    return out


def run_batch(args):
    """The 256-mesh uneven batch (triangles p = 1..6, tetrahedra p = 1..5, cell
    counts log-uniform in 1e3..2e5, seed 6): one graph replay of fe_batch_run =
    factor + persistent element launch over every mesh's tiles + one assembly
    launch over every mesh's rows, BF16.  Reports element matrices/s (both
    forms), nnz/s and the achieved fraction of the per-mesh roofline
    sum_m max(bytes_m / HBM, flops_m / BF16 peak)."""
    import torch
    from paper_2410_12614_gb300 import api, inputs
    stream = torch.cuda.Stream()
    plans, kaps = [], []
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i, x in enumerate(inputs.batched_workload()):
            v, c = inputs.structured_mesh(x["cell_type"], x["n"], x["alpha"], x["seed"])
            pts, w = api.quadrature_rule(x["cell_type"], x["degree"] + 1)
            plan = api.Plan(x["cell_type"], v, c, x["degree"], pts, w, precisions=("bf16",), stream=stream)
            plans.append(plan)
            kaps.append(torch.from_numpy(inputs.lognormal_kappa(plan.n_cells, plan.n_q, 500 + i)).cuda())
        setup_s = time.perf_counter() - t0
        batch = api.Batch(plans, kaps, prec="bf16", stream=stream)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        sink = torch.empty((), dtype=torch.float32, device="cuda")
        for _ in range(2):
            batch.run()
        batch.sync()
        times = []
        for _ in range(max(3, args.steps // 2)):
            flush.fill_(1.0)
            sink.copy_(flush.sum())
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.run()
            e1.record(stream)
            stream.synchronize()
            times.append(e0.elapsed_time(e1))
        batch.sync()
    ms = statistics.median(times)
    hbm, _ = _peaks()
    peak_tf = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
    ideal = 0.0
    n_cells = nnz = 0
    for p in plans:
        fb, eb, ab = algorithmic_bytes(p, "bf16")
        n_sym = p.n_phi * (p.n_phi + 1) // 2
        pairs = p.d * (p.d + 1) // 2
        flops = 2.0 * p.n_cells * p.n_q * (pairs + 1) * n_sym
        ideal += max((fb + eb + ab) / (hbm * 1e9), flops / (peak_tf * 1e12))
        n_cells += p.n_cells
        nnz += p.nnz
    return {"meshes": len(plans), "cells": n_cells, "nnz_per_matrix": nnz, "ms_per_run": ms,
            "element_matrices_per_s": 2 * n_cells / (ms / 1e3), "nnz_per_s": 2 * nnz / (ms / 1e3),
            "ideal_ms": ideal * 1e3, "frac_of_roofline": ideal * 1e3 / ms, "launches": batch.launches,
            "plan_setup_s": setup_s}


_POOL_STATE = {}


def _pool_init():
    """Worker set-up: rebuild the seeded workload and the oracle problem."""
    import oracle
    from paper_2410_12614_gb300 import inputs
    v, c = make_inputs()
    pts, w = oracle.collapsed_rule("tetrahedron", DEGREE + 1)
    ref = oracle.Problem(v, c, DEGREE, pts, w)
    _POOL_STATE["ref"] = ref
    _POOL_STATE["kap"] = inputs.lognormal_kappa(ref.n_cells, ref.n_q, SEED_KAPPA)


def _pool_task(ids):
    ref, kap = _POOL_STATE["ref"], _POOL_STATE["kap"]
    return {f: ref.element_matrices_subset(kap, f, ids) for f in ("stiffness", "mass")}


def cpu_baseline_all_cores(budget_s, per_cell_1core):
    """The same oracle on every host core (one spawned process per core, each
    computing both forms for a slice of a random cell sample; the parent then
    assembles the sample into the CSR values), inside a bounded time budget."""
    import multiprocessing as mp
    import oracle
    cores = os.cpu_count() or 1
    v, c = make_inputs()
    pts, w = oracle.collapsed_rule("tetrahedron", DEGREE + 1)
    ref = oracle.Problem(v, c, DEGREE, pts, w)
    ref.csr_pattern()
    n = int(max(cores * 64, min(ref.n_cells, cores * budget_s / max(per_cell_1core, 1e-9))))
    rng = np.random.default_rng(98)
    ids = np.sort(rng.choice(ref.n_cells, size=n, replace=False))
    parts = np.array_split(ids, cores * 4)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_pool_init) as pool:
        pool.map(_pool_task, [p[:8] for p in parts[:cores]])   # warm every worker
        t0 = time.perf_counter()
        res = pool.map(_pool_task, parts)
        for f in ("stiffness", "mass"):
            ref.assemble_subset(np.concatenate([r[f] for r in res]), ids)
        dt = time.perf_counter() - t0
    return {"value": 2 * n / dt, "unit": "element matrices/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} random cells of the workload, both forms, {cores} spawned processes; "
                      "assembled into the CSR values by the parent", "seconds": dt}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    budget = getattr(args, "ref_budget_s", None) or max(2.0, min(30.0, 120.0 / max(1, args.steps + args.warmup)))
    times, val = [], None
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(args, budget_s=budget)
        if i >= args.warmup:
            times.append(r)
    value = statistics.mean(t["value"] for t in times)
    ms = 2 * 82944 / value * 1e3
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value, "unit": "element matrices/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded structured mesh + lognormal kappa)",
        "config": workload_config(world),
        "method": "the FP64 CPU oracle (literal quadrature loops, cell-order assembly) on a bounded random "
                  "cell sample of the workload per step, single-threaded",
        "cpu_baseline": {"value": value, "unit": "element matrices/s", "cores": 1, "kind": "oracle",
                         "sample": times[-1]["sample"]},
        "e2e": {"value": value, "unit": "element matrices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--with-batch", action="store_true",
                    help="also time the 256-mesh uneven batch (adds about a minute of plan set-up)")
    ap.add_argument("--sweep", action="store_true",
                    help="also time the element kernels for P1..P8 tetrahedra on 16^3 x 6 in every precision")
    ap.add_argument("--configs", action="store_true",
                    help="also time P1 Laplace FP64 (2,048 triangles) and the P2 adjoint on 196,608 tetrahedra")
    ap.add_argument("--configs-only", action="store_true", help="time only those two configurations")
    ap.add_argument("--sweep-only", action="store_true",
                    help="time only the degree sweep and print it as the JSON line (a profiling entry point)")
    ap.add_argument("--boxed-sweep", action="store_true", help="Q_p hexahedra against FP64 (--boxed-degrees)")
    ap.add_argument("--boxed-degrees", default="1,2,3,4,5")
    ap.add_argument("--boxed-only", action="store_true", help="time only the boxed sweep (a profiling entry point)")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the compact context lines (sweep points, Q3 hexahedra, small configurations)")
    ap.add_argument("--sweep-degrees", default="1,2,3,4,5,6,7,8")
    ap.add_argument("--sweep-precisions", default="bf16,fp16,tf32,tf32x3,e4m3,fp64")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.configs_only:
        if rank == 0:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            print(json.dumps({"small_configs": run_configs(args)}))
        return
    if args.boxed_only:
        if rank == 0:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            print(json.dumps({"boxed_sweep": run_boxed_sweep(args)}))
        return
    if args.sweep_only:
        if rank == 0:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            print(json.dumps({"degree_sweep": run_sweep(args)}))
        return
    res = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
