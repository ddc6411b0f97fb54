#!/usr/bin/env python
"""Throughput of randomized CUR-ID (Algorithms 3 + 4) on one GB300.

Workload (seeded, synthetic, resident in HBM): dense float32 A of
8000 x 6000 = U_a diag(sigma) V_a^T with sigma_j = j^-2 and Haar factors;
rank k = 200, oversampling p = 10, one power step (q = 1); a fresh Gaussian
Omega (210 x 8000) is drawn on the device every step from the step's seed.
One step = Omega, the three products with A, two row orthonormalisations,
CPQR of Y (210 x 6000), T, the gather of C, the full CPQR of C^T
(200 x 8000), the gather of R and U = V* R^+ -- the whole decomposition.
A (192 MB) is larger than the 129 MB L2, so no flush is needed between steps.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (the reference arm of this comparison).
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "rank-k CUR/ID decompositions/sec at stated rel. error; % of HBM/TC roofline"
UNIT = "decompositions/s"
M, N, K, P, Q = 8000, 6000, 200, 10, 1
BASE_SEED = 1413
FP32_FMA_PER_SM_CLK = 128          # FP32 lanes per SM
# dram__bytes_read.sum + dram__bytes_write.sum of one cpqr_reg_kernel launch on
# this workload from the ncu capture named below (empty: no capture of the
# current kernel yet)
CPQR_DRAM_BYTES = {"cpqr_col": 5.142e6 + 18.4e3, "cpqr_row": 6.695e6 + 24.3e3}
CPQR_DRAM_SOURCE = ("profiles/cpqr_reg_kernel_randomized_cur_f32_8000x6000_k200.md "
                    "(ncu dram__bytes_read.sum + dram__bytes_write.sum of the one-at-a-time "
                    "cpqr_reg_kernel<float, 7, 4, 16> launches)")
NUM_SMS = 152


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=M)
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--k", type=int, default=K)
    ap.add_argument("--p", type=int, default=P)
    ap.add_argument("--q", type=int, default=Q)
    ap.add_argument("--tf32", type=int, default=1)
    ap.add_argument("--inflight", type=int, default=8,
                    help="decompositions in flight (one stream and workspace each)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--only-form", choices=["adjoint", "batched", "mixed", "srft", "sparse", "extras",
                                                "c1"], default=None,
                    help="run only this form's measurement and print its JSON")
    ap.add_argument("--small", action="store_true",
                    help="with --only-form: profiling sizes (256 blocks; BF16 8192^2, q = 1)")
    return ap.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device):
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms during a region."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.remove(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpqr_flops(m, n, k):
    """Algorithmic flops of a rank-k Householder CPQR of an m x n matrix
    (the cost model of Section 4): 4 [m n k - (m + n) k^2 / 2 + k^3 / 3]."""
    return 4.0 * (m * n * k - (m + n) * k * k / 2.0 + k ** 3 / 3.0)


def phase_work(args, l):
    """Algorithmic flops / bytes per launch of the main kernels (float32)."""
    m, n, k = args.m, args.n, args.k
    return {
        # one product with A (the sketch phase times each of the 2q + 1
        # products as one call): 2 l m n flops, A read once
        "sketch": {"flops": 2.0 * l * m * n, "bytes": 4.0 * (m * n + l * max(m, n) * 2)},
        # CPQR of Y (l x n, k steps) and of C^T (k x m, k steps)
        "cpqr_col": {"flops": cpqr_flops(l, n, k), "bytes": 4.0 * (l * n + k * n + n)},
        "cpqr_row": {"flops": cpqr_flops(k, m, k), "bytes": 4.0 * (2 * k * m + m)},
    }


def rel_err_gpu(A, J, I, U, k):
    """||A - C U R||_F / ||A||_F in float64 on the GPU, C = A(:, J[:k]),
    R = A(I[:k], :)."""
    Ad = A.double()
    C = Ad[:, J[:k].long()]
    R = Ad[I[:k].long(), :]
    return float(torch.linalg.norm(Ad - (C @ U.double()) @ R) / torch.linalg.norm(Ad))


def run_ours(args, ws, rank, local):
    import paper_1412_8447_gb300 as curid
    from paper_1412_8447_gb300.build import build
    import synthetic as syn

    if rank == 0:
        build()
    barrier(ws)
    if ws > 1:
        build()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    l = args.k + args.p
    A = syn.spectrum_matrix(args.m, args.n, syn.power_decay(min(args.m, args.n)),
                            BASE_SEED + rank, torch.float32, dev)
    tf32 = bool(args.tf32)
    kin = max(1, args.inflight)
    main = torch.cuda.current_stream(dev)
    # one stream and one library handle (slot) per decomposition in flight
    streams = [main] + [torch.cuda.Stream(dev) for _ in range(kin - 1)]
    outs = []
    for s in range(kin):
        with torch.cuda.stream(streams[s]), curid.inflight(s):
            outs.append(curid.cur_outputs(A, args.k))

    def step(i, slot=None):
        s = i % kin if slot is None else slot
        with torch.cuda.stream(streams[s]), curid.inflight(s):
            curid.cur(A, args.k, p=args.p, q=args.q, seed=BASE_SEED * 1000 + i, tf32=tf32,
                      out=outs[s], check=False)

    def slot_status(s):
        with torch.cuda.stream(streams[s]), curid.inflight(s):
            return curid.last_status(local)

    def check_status(where, slots):
        for s in range(slots):
            st, _ = slot_status(s)
            if st not in (0, 2):
                raise RuntimeError(f"device status {curid.STATUS_NAMES[st]} in {where}")

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # ---- 1. one decomposition at a time: latency, per-phase times and the
    # launch durations the roofline uses (kernels timed in isolation) --------
    curid.set_concurrency(1, local)
    for i in range(args.warmup):
        step(i, 0)
    check_status("warm-up", 1)
    curid.profile(True, local)
    lat_steps = max(5, min(args.steps, 10))
    torch.cuda.synchronize(dev)
    e0.record(main)
    for i in range(lat_steps):
        step(args.warmup + i, 0)
    e1.record(main)
    torch.cuda.synchronize(dev)
    lat_ms = e0.elapsed_time(e1) / lat_steps
    phase_ms, phase_calls, lat_launches = curid.profile_read(local)
    curid.profile(False, local)
    # accuracy of the decomposition whose Omega the oracle uses below
    step(0, 0)
    torch.cuda.synchronize(dev)
    err_gpu = rel_err_gpu(A, outs[0].J, outs[0].I, outs[0].U, args.k)

    # ---- 2. throughput: kin decompositions in flight, K timed steps ---------
    for s in range(kin):
        with torch.cuda.stream(streams[s]), curid.inflight(s):
            curid.set_concurrency(kin, local)
    for i in range(max(args.warmup, 2 * kin)):
        step(1000 + i)
    torch.cuda.synchronize(dev)
    check_status("warm-up", kin)
    for s in range(kin):
        with torch.cuda.stream(streams[s]), curid.inflight(s):
            curid.profile(True, local)
            curid.profile_read(local)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier(ws)
    torch.cuda.synchronize(dev)
    e0.record(main)
    for st in streams[1:]:
        st.wait_event(e0)
    for i in range(args.steps):
        step(2000 + i)
    for st in streams[1:]:
        main.wait_stream(st)
    e1.record(main)
    torch.cuda.synchronize(dev)
    barrier(ws)
    elapsed_ms = e0.elapsed_time(e1)
    launches = 0
    for s in range(kin):
        with torch.cuda.stream(streams[s]), curid.inflight(s):
            launches += curid.profile_read(local)[2]
            curid.profile(False, local)
    clk = clocks.stop()
    check_status("timed region", kin)
    elapsed_ms = max_over_ranks(elapsed_ms, ws, dev)
    value = args.steps * ws / (elapsed_ms / 1e3)

    # end to end through the public API with host buffers: every step copies
    # its matrix from pinned host memory and its (J, I, U) back; HostStream
    # keeps kin decompositions in flight and overlaps the copies with them
    e2e = None
    if not args.no_e2e:
        A_host = A.cpu().pin_memory()
        ke = max(2 * kin, min(args.steps, 12))
        hs = curid.HostStream(args.m, args.n, args.k, A.dtype, local, p=args.p, q=args.q,
                              tf32=tf32, inflight=kin)
        res = hs.host_results(ke)
        seeds = [BASE_SEED * 1000 + 7000 + i for i in range(ke)]
        hs.run([A_host] * ke, res, seeds)
        torch.cuda.synchronize(dev)
        barrier(ws)
        e0.record(main)
        hs.run([A_host] * ke, res, seeds)
        e1.record(main)
        torch.cuda.synchronize(dev)
        e2e_ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
        e2e = {"value": ke * ws / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": A.numel() * 4,
               "d2h_bytes_per_step": (args.n + args.m) * 4 + args.k * args.k * 8,
               "steps": ke,
               "how": f"HostStream: {kin} decompositions in flight on {kin} streams, the copy "
                      "of the next matrices on three side streams"}
        del hs

    pk, pk_kind = peaks()
    work = phase_work(args, l)
    per_step = {p: phase_ms[p] / lat_steps for p in phase_ms}
    total_phase = sum(phase_ms.values()) or 1.0
    fam = {"cpqr": ("cpqr_col", "cpqr_row"), "sketch": ("sketch",),
           "orth": ("orth",), "u_solve": ("u_solve",)}
    fam_ms = {f: sum(phase_ms[p] for p in ps) for f, ps in fam.items()}
    dominant = max(fam_ms, key=fam_ms.get)
    sm_mhz_max = clk["sm_max_mhz"] or 2070.0
    fp32_peak = NUM_SMS * FP32_FMA_PER_SM_CLK * 2 * sm_mhz_max * 1e6 / 1e12
    fp32_src = "derived: 152 SMs x 128 FP32 FMA/clk x 2 x max SM clock"

    def sketch_roof():
        calls = phase_calls["sketch"]
        if not calls:
            return None
        dur_s = phase_ms["sketch"] / calls / 1e3
        ach = work["sketch"]["flops"] / dur_s / 1e12
        if tf32:
            peak = pk["bf16_tflops_sustained"] / 2
            return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None,
                    "hbm_frac": work["sketch"]["bytes"] / dur_s / 1e9 / pk["hbm_gbs"],
                    "kernel": "tc_sketch_kernel (tcgen05 TF32, A split hi + lo: 2 MMAs per "
                              "K step; achieved counts each product once)",
                    "peak_source": f"{pk_kind} bf16 sustained x 1/2 (TF32 nominal ratio)"}
        return {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": None, "kernel": "gemm_simt_kernel (FP32 FMA)",
                "peak_source": fp32_src}

    roof = None
    if dominant == "cpqr":
        calls = phase_calls["cpqr_col"] + phase_calls["cpqr_row"]
        if calls:
            flops = (work["cpqr_col"]["flops"] * phase_calls["cpqr_col"]
                     + work["cpqr_row"]["flops"] * phase_calls["cpqr_row"])
            ach = flops / (fam_ms["cpqr"] / 1e3) / 1e12
            default = (args.m, args.n, args.k, args.p) == (M, N, K, P)
            traffic = ((CPQR_DRAM_BYTES["cpqr_col"] * phase_calls["cpqr_col"]
                        + CPQR_DRAM_BYTES["cpqr_row"] * phase_calls["cpqr_row"]) / calls
                       if default and CPQR_DRAM_BYTES else None)
            roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": ach / fp32_peak, "traffic": traffic,
                    "traffic_source": CPQR_DRAM_SOURCE if traffic else None,
                    "algorithmic_flops_per_launch": flops / calls,
                    "algorithmic_bytes": (work["cpqr_col"]["bytes"] * phase_calls["cpqr_col"]
                                          + work["cpqr_row"]["bytes"] * phase_calls["cpqr_row"])
                                         / calls,
                    "launch_ms": fam_ms["cpqr"] / calls,
                    "kernel": f"cpqr_reg_kernel (CPQR of Y {l}x{args.n} and of C^T {args.k}x"
                              f"{args.m}, {args.k} steps each, flops 4[mnk - (m+n)k^2/2 + k^3/3]; "
                              f"timed one decomposition at a time; bound by the per-step "
                              f"grid-wide pivot exchange, not by FP32 rate)",
                    "peak_source": fp32_src}
    elif dominant == "sketch":
        roof = sketch_roof()
    else:
        roof = {"bound": "alu", "achieved": None, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": None, "traffic": None,
                "kernel": f"{dominant} (chain of small kernels; no single-kernel figure)",
                "peak_source": fp32_src}
    cpu = None
    err_oracle = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, err_oracle = cpu_baseline(args, A, curid)
    # the forms below run one decomposition at a time: put back the handles'
    # concurrency (the in-flight passes set it on every slot)
    for s in range(kin):
        with torch.cuda.stream(streams[s]), curid.inflight(s):
            curid.set_concurrency(1, local)
    forms = None
    if rank == 0 and ws == 1 and not args.no_forms:
        forms = {"adjoint": measure_adjoint(dev), "batched": measure_batched(dev),
                 "mixed": measure_mixed(dev), "srft": measure_srft(dev),
                 "sparse": measure_sparse(dev), "c1": measure_c1(dev)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "tf32+f32" if tf32 else "f32",
        "data": "synthetic (seeded; sigma_j = j^-2, Haar factors; Omega drawn on device)",
        "config": {"workload": f"randomized CUR-ID, float32 A {args.m}x{args.n}, k={args.k}, "
                               f"p={args.p}, q={args.q}, Omega {l}x{args.m}",
                   "m": args.m, "n": args.n, "k": args.k, "p": args.p, "q": args.q,
                   "inflight": kin,
                   "l2": "inputs larger than L2 (A is %.0f MB), no flush" % (A.numel() * 4 / 1e6),
                   "parallelism": f"replicas x{ws}; {kin} decompositions in flight per GPU "
                                  f"(one stream and workspace each)"},
        "latency_ms": lat_ms,
        "accuracy": {"rel_err_fro": err_gpu, "oracle_rel_err_fro": err_oracle,
                     "abs_diff": (abs(err_gpu - err_oracle) if err_oracle is not None else None),
                     "how": f"||A - CUR||_F / ||A||_F in float64 for the decomposition with "
                            f"seed {BASE_SEED * 1000}; the oracle runs the same Omega"},
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                   "reasons": clk["reasons"], "samples": clk["samples"]},
        "e2e": e2e, "gpu_launches": launches,
        "roofline": roof,
        "sketch_roofline": sketch_roof(),
        "phases_ms_per_step": {p: round(v, 4) for p, v in per_step.items()},
        "phase_share": {p: round(phase_ms[p] / total_phase, 4) for p in phase_ms},
        "launches_per_decomposition": lat_launches / lat_steps,
        "cpu_baseline": cpu,
        "forms": forms,
    }
    if rank == 0:
        print(json.dumps(line))


def measure_adjoint(dev, steps=10, warmup=3):
    """Forward + backward of the differentiable CUR-ID (skeletons frozen) on
    A 2048 x 1024, sigma_j = exp(-j/20), k = 64, deterministic, loss
    1/2 ||A - C U R||_F^2 in the dtype of A; float32 and the plain float64
    GPU path, CUDA events on the current stream."""
    import paper_1412_8447_gb300 as curid
    import synthetic as syn
    m, n, k = 2048, 1024, 64
    stream = torch.cuda.current_stream(dev)
    res = {"workload": f"differentiable CUR-ID, A {m}x{n}, sigma_j = exp(-j/20), k = {k}, "
                       "deterministic; loss 1/2 ||A - CUR||_F^2, forward + backward through "
                       "the library adjoint (skeletons frozen)",
           "unit": "forward+backward/s"}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        A0 = syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 20.0), BASE_SEED + 5, dt, dev)

        def step():
            A = A0.detach().requires_grad_(True)
            C, U, R, _, _ = curid.cur_differentiable(A, k)
            Res = A - C @ (U.to(dt) @ R)
            loss = 0.5 * (Res * Res).sum()
            loss.backward()
            return A.grad

        for _ in range(warmup):
            step()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        res[name] = {"value": 1e3 / ms, "ms_per_step": ms}
    res["f32_over_f64"] = res["f32"]["value"] / res["f64"]["value"]
    # algorithmic work of one forward + backward: the cost model of Section 4
    # for the two CPQRs, T and U, and six m x n x k products for the adjoint
    fwd = (cpqr_flops(m, n, k) + cpqr_flops(k, m, k) + float(k) * k * (n - k)
           + 6.0 * k * k * n)
    bwd = 6 * 2.0 * m * n * k
    peak = NUM_SMS * FP32_FMA_PER_SM_CLK * 2 * 2070e6 / 1e12
    ach = (fwd + bwd) / (res["f32"]["ms_per_step"] / 1e3) / 1e12
    res["roofline"] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                       "frac": ach / peak, "flops_per_step": fwd + bwd,
                       "peak_source": "derived FP32: 152 SMs x 128 FMA/clk x 2 x 2070 MHz",
                       "note": "latency-bound: about 40 dependent launches per step"}
    return res


def measure_c1(dev, reps=20, inflight=8, steps=64):
    """The small deterministic workload: CUR-ID of a float64 400 x 300
    matrix (sigma_j = exp(-j/10), Haar factors), k = 40, no sketch: latency
    of one call (median of single calls, CUDA events), throughput with
    `inflight` decompositions in flight (one stream and workspace each), the
    FP64 rate achieved on the cost model of Section 4, and the error against
    the FP64 oracle."""
    import oracle as O
    import paper_1412_8447_gb300 as curid
    import synthetic as syn
    m, n, k = 400, 300, 40
    A = syn.spectrum_matrix(m, n, syn.exp_decay(min(m, n), 10.0), BASE_SEED, torch.float64, dev)
    main = torch.cuda.current_stream(dev)
    streams = [main] + [torch.cuda.Stream(dev) for _ in range(inflight - 1)]
    outs = []
    for s in range(inflight):
        with torch.cuda.stream(streams[s]), curid.inflight(s):
            curid.set_concurrency(inflight, dev.index or 0)
            outs.append(curid.cur_outputs(A, k))

    def call(s):
        with torch.cuda.stream(streams[s]), curid.inflight(s):
            curid.cur(A, k, out=outs[s], check=False)

    for s in range(inflight):
        call(s)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat = []
    curid.set_concurrency(1, dev.index or 0)
    call(0)
    for _ in range(reps):
        e0.record(main)
        call(0)
        e1.record(main)
        torch.cuda.synchronize(dev)
        lat.append(e0.elapsed_time(e1))
    curid.set_concurrency(inflight, dev.index or 0)
    e0.record(main)
    for st in streams[1:]:
        st.wait_event(e0)
    for i in range(steps):
        call(i % inflight)
    for st in streams[1:]:
        main.wait_stream(st)
    e1.record(main)
    torch.cuda.synchronize(dev)
    thr = steps / (e0.elapsed_time(e1) / 1e3)
    flops = (cpqr_flops(m, n, k) + cpqr_flops(k, m, k) + float(k) * k * (n - k)
             + 2.0 * k * k * n + 4.0 * k * k * n)
    Ah = A.cpu().numpy()
    o = O.cur(Ah, k)
    eg = rel_err_gpu(A, outs[0].J, outs[0].I, outs[0].U, k)
    eo = O.rel_err_fro(Ah, o.C, o.U, o.R)
    return {"workload": f"deterministic CUR-ID, float64 A {m}x{n}, sigma_j = exp(-j/10), "
                        f"k = {k}", "unit": "decompositions/s",
            "latency_ms": statistics.median(lat), "value": thr, "inflight": inflight,
            "flops_per_decomposition": flops,
            "fp64_tflops": flops * thr / 1e12, "fp64_peak_tflops": 1.25,
            "fp64_frac": flops * thr / 1e12 / 1.25,
            "peak_source": "nominal GB300 FP64 1.25 TFLOP/s",
            "rel_err_fro": eg, "oracle_rel_err_fro": eo, "same_skeleton":
                bool(list(outs[0].J[:k].cpu().tolist()) == list(o.J[:k])
                     and list(outs[0].I[:k].cpu().tolist()) == list(o.I[:k]))}


def measure_batched(dev, replays=5, nb=4096):
    """Batched adaptive-rank column ID of 4096 Laplace blocks (m_b, n_b
    uniform on 64..512): autotuned launch shape, the launch captured in a
    CUDA graph and replayed; float64 (tol 1e-8) and float32 (tol 1e-5).  The
    plain float64 GPU path (one adaptive curid_cpqr call per block) is timed
    on 64 of the blocks for comparison."""
    import paper_1412_8447_gb300 as curid
    import synthetic as syn
    stream = torch.cuda.current_stream(dev)
    res = {"workload": f"batched adaptive-rank column ID, {nb} Laplace blocks 1/|x-y| "
                       "(unit boxes 3 apart), m_b, n_b uniform on 64..512, one persistent "
                       "launch replayed from a CUDA graph",
           "unit": "blocks/s"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, dt, tol, peak, src in (
            ("f64", torch.float64, 1e-8, 1.25, "nominal FP64 1.25 TFLOP/s"),
            ("f32", torch.float32, 1e-5, NUM_SMS * FP32_FMA_PER_SM_CLK * 2 * 2070e6 / 1e12,
             "derived FP32 peak")):
        flat, shapes, offs = syn.laplace_batch(nb, BASE_SEED + 4, dt, dev)
        B = curid.BatchedID(flat, shapes, offs, tol=tol, k_max=64)
        threads, per_sm = B.autotune()
        B.run()
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            B.run()
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(replays):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / replays
        k = B.k_out.cpu().tolist()
        flops = sum(cpqr_flops(m, n, kb) + float(kb) * kb * (n - kb)
                    for (m, n), kb in zip(shapes, k))
        ach = flops / (ms / 1e3) / 1e12
        entry = {"value": nb / (ms / 1e3), "ms_per_batch": ms, "tol": tol,
                 "launch_shape": {"threads": threads, "ctas_per_sm": per_sm},
                 "mean_rank": sum(k) / nb, "max_rank": max(k),
                 "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                              "frac": ach / peak, "peak_source": src}}
        if name == "f64":
            sample = list(range(0, nb, nb // 64))[:64]
            plain = []
            for b in sample:
                m, n = shapes[b]
                plain.append(flat[offs[b]:offs[b] + m * n].view(m, n))
            curid.cpqr(plain[0], tol=tol)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for Ab in plain:
                curid.cpqr(Ab, tol=tol, check=False)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            pms = e0.elapsed_time(e1) / len(plain)
            entry["plain_f64_path"] = {"value": 1e3 / pms, "unit": "blocks/s",
                                       "how": "one adaptive curid_cpqr launch per block, "
                                              "64 sampled blocks (T solve not included)"}
        res[name] = entry
        del B, g, flat
        torch.cuda.empty_cache()
    return res


def measure_mixed(dev, steps=3, size=20000, q=None, with_f64=True):
    """Precision form at A 20000 x 20000 stored in bfloat16, sigma_j =
    10^(-6j/500) (j <= 500), floor 1e-7, k = 500, p = 20, q = 2: the BF16
    tensor-core path against the plain float64 GPU path on the same values
    (one timed run of the latter), both with errors ||A - CUR||_F / ||A||_F
    computed in float64 on the GPU."""
    import paper_1412_8447_gb300 as curid
    import synthetic as syn
    w = syn.workload_mixed_bf16(device=dev, m=size, n=size)
    A, k, p = w["A"], w["k"], w["p"]
    q = w["q"] if q is None else q
    m, n = A.shape
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def err(X, r):
        Xd = X.double()
        D = Xd - (r.C.double() @ r.U) @ r.R.double()
        return float(torch.linalg.norm(D) / torch.linalg.norm(Xd))

    def timed(X, nrep, seed0):
        out = curid.cur_outputs(X, k, want_c=True, want_r=True)
        curid.cur(X, k, p=p, q=q, seed=seed0, out=out)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for i in range(nrep):
            curid.cur(X, k, p=p, q=q, seed=seed0 + 1 + i, out=out, check=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        st, _ = curid.last_status(dev.index or 0)
        return e0.elapsed_time(e1) / nrep, out, st

    res = {"workload": f"randomized CUR-ID, A {m}x{n} stored in bfloat16, sigma_j = "
                       f"10^(-6j/500) (j <= 500), floor 1e-7, k = {k}, p = {p}, q = {q}",
           "unit": "decompositions/s"}
    ms, out, st = timed(A, steps, 7000)
    curid.profile(True, dev.index or 0)
    curid.cur(A, k, p=p, q=q, seed=6999, out=out, check=False)
    phase_ms, _, launches = curid.profile_read(dev.index or 0)
    curid.profile(False, dev.index or 0)
    flops = (2 * q + 1) * 2.0 * (k + p) * m * n
    res["bf16"] = {"value": 1e3 / ms, "ms_per_step": ms, "status": curid.STATUS_NAMES[st],
                   "rel_err_fro": err(A, out),
                   "phases_ms": {ph: round(v, 3) for ph, v in phase_ms.items()},
                   "launches": launches,
                   "products_tflops": flops / (sum(v for ph, v in phase_ms.items()
                                                   if ph == "sketch") / 1e3) / 1e12}
    if not with_f64:
        return res
    A64 = A.double()
    ms64, out64, st64 = timed(A64, 1, 7000)
    res["f64_plain"] = {"value": 1e3 / ms64, "ms_per_step": ms64,
                        "status": curid.STATUS_NAMES[st64], "rel_err_fro": err(A64, out64),
                        "how": "the same pipeline in float64 (SIMT products), one timed run"}
    res["bf16_over_f64"] = res["bf16"]["value"] / res["f64_plain"]["value"]
    del A64, out64
    torch.cuda.empty_cache()
    return res


def measure_srft(dev, steps=10, m=M, n=N, k=K):
    """Accelerated randomized scheme (Section 5.2): the structured Omega of
    Eq. (5.2) (real form: DCT-II rows with random signs, rows and signs drawn
    on the device each step), l = 2k, no power step, on the benchmark matrix.
    "srft": Omega A by the fast transform (Omega never formed), U = V* R^+;
    "srft_corrected_u": the same with the error-corrected U of Eq. (4.3);
    "srft_explicit": Omega formed and applied by the TF32 tensor-core product;
    "gaussian_same_l": a Gaussian Omega with the same l, TF32 product.
    "sample_ms": the sample Y = Omega A alone, fast transform against the
    formed Omega's TF32 product.  Errors ||A - CUR||_F / ||A||_F in float64
    on the GPU."""
    import paper_1412_8447_gb300 as curid
    import synthetic as syn
    l = 2 * k
    A = syn.spectrum_matrix(m, n, syn.power_decay(min(m, n)), BASE_SEED, torch.float32, dev)
    out = curid.cur_outputs(A, k, want_c=True, want_r=True)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def err():
        Ad = A.double()
        D = Ad - (out.C.double() @ out.U) @ out.R.double()
        return float(torch.linalg.norm(D) / torch.linalg.norm(Ad))

    def srft_step(i):
        rows, signs = curid.srft_draw(m, l, 5000 + i, device=dev.index or 0)
        curid.cur(A, k, p=l - k, q=0, omega=curid.Srft(rows, signs), tf32=True, out=out,
                  check=False)

    def srft_corrected_step(i):
        rows, signs = curid.srft_draw(m, l, 5000 + i, device=dev.index or 0)
        curid.cur(A, k, p=l - k, q=0, omega=curid.Srft(rows, signs), tf32=True, out=out,
                  check=False, corrected=True)

    def srft_explicit_step(i):
        rows, signs = curid.srft_draw(m, l, 5000 + i, device=dev.index or 0)
        Om = curid.srft_omega(rows, signs, torch.float32)
        curid.cur(A, k, p=l - k, q=0, omega=Om, tf32=True, out=out, check=False)

    def gauss_step(i):
        curid.cur(A, k, p=l - k, q=0, seed=6000 + i, tf32=True, out=out, check=False)

    res = {"workload": f"randomized CUR-ID, float32 A {m}x{n}, sigma_j = j^-2, k = {k}, "
                       f"l = 2k = {l}, q = 0, TF32 products",
           "unit": "decompositions/s"}
    for name, fn in (("srft", srft_step), ("srft_corrected_u", srft_corrected_step),
                     ("srft_explicit", srft_explicit_step), ("gaussian_same_l", gauss_step)):
        for i in range(3):
            fn(i)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for i in range(steps):
            fn(10 + i)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        st, _ = curid.last_status(dev.index or 0)
        res[name] = {"value": 1e3 / ms, "ms_per_step": ms, "status": curid.STATUS_NAMES[st],
                     "rel_err_fro": err()}
    # the sample alone: the fast transform against the formed Omega's product
    rows, signs = curid.srft_draw(m, l, 7000, device=dev.index or 0)
    Om = curid.srft_omega(rows, signs, torch.float32)
    sample = {}
    for name, fn in (("fast", lambda: curid.srft_sketch(A, rows, signs)),
                     ("explicit_tf32", lambda: curid.sketch_matrix(A, Om, q=0, tf32=True))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sample[name] = e0.elapsed_time(e1) / steps
    sample["fast_hbm_gbs"] = m * n * 4 / (sample["fast"] * 1e-3) / 1e9
    res["sample_ms"] = sample
    del A, out
    torch.cuda.empty_cache()
    return res


def measure_sparse(dev, steps=5, m=300000, n=300, k=40, p=10, q=2):
    """Sparse input (Section 1's case for CUR): a sum of 300 sparse
    non-negative rank-one terms shaped like A_1 of Section 6 (300000 x 300,
    about 1.07M stored entries, float32), randomized CUR-ID with k = 40,
    p = 10, q = 2 through the sparse path, against the dense path (TF32
    tensor-core products) on the same values.  Errors ||A - CUR||_F / ||A||_F
    in float64 on the GPU."""
    import paper_1412_8447_gb300 as curid
    import synthetic as syn
    As = syn.sparse_rank_sum(m, n, syn.a1_coeffs(), BASE_SEED + 5)
    A = syn.to_torch_csr(As, torch.float32, dev)
    Ad = torch.tensor(As.toarray(), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def err(r):
        X = Ad.double()
        D = X - (r.C.double() @ r.U) @ r.R.double()
        return float(torch.linalg.norm(D) / torch.linalg.norm(X))

    res = {"workload": f"randomized CUR-ID of a sparse A {m}x{n} (sum of 300 sparse rank-one "
                       f"terms, {As.nnz} stored entries), k = {k}, p = {p}, q = {q}",
           "unit": "decompositions/s"}
    runs = (("sparse", lambda i, out: curid.cur_sparse(A, k, p, q=q, seed=9000 + i, out=out,
                                                       check=False)),
            ("dense_tf32", lambda i, out: curid.cur(Ad, k, p=p, q=q, seed=9000 + i, tf32=True,
                                                    out=out, check=False)))
    for name, fn in runs:
        out = curid.cur_outputs(Ad, k, want_c=True, want_r=True)
        for i in range(2):
            fn(i, out)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for i in range(steps):
            fn(10 + i, out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        st, _ = curid.last_status(dev.index or 0)
        res[name] = {"value": 1e3 / ms, "ms_per_step": ms, "status": curid.STATUS_NAMES[st],
                     "rel_err_fro": err(out)}
    res["sparse_over_dense"] = res["sparse"]["value"] / res["dense_tf32"]["value"]
    del A, Ad
    torch.cuda.empty_cache()
    return res


def measure_extras(dev, steps=5):
    """Rows measured on request (``--only-form extras``): the adaptive rank
    with a sketch (benchmark matrix, tol 1e-3, p = 10, q = 1, TF32: time per
    call including its sample-size search), complex A (2000 x 1500
    complex64 with sigma_j = j^-2, k = 100, p = 10, q = 1, through the real
    embedding) against the real path on the real part, and the two
    stabilised T solves (k = 200, n = 6000)."""
    import paper_1412_8447_gb300 as curid
    import synthetic as syn
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, n=steps):
        fn()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / n

    res = {}
    A = syn.spectrum_matrix(M, N, syn.power_decay(N), BASE_SEED, torch.float32, dev)
    r = curid.cur(A, 0, p=10, q=1, seed=3, tf32=True, tol=1e-3, want_c=True, want_r=True)
    ms = timed(lambda: curid.cur(A, 0, p=10, q=1, seed=3, tf32=True, tol=1e-3))
    Ad = A.double()
    e = float(torch.linalg.norm(Ad - (r.C.double() @ r.U) @ r.R.double()) / torch.linalg.norm(Ad))
    res["adaptive_sketch"] = {"workload": f"float32 A {M}x{N}, sigma_j = j^-2, tol 1e-3, p = 10, "
                                          f"q = 1, TF32", "ms_per_call": ms, "k": r.k,
                              "rel_err_fro": e}
    del Ad, r
    m, n, k = 2000, 1500, 100
    Ar = syn.spectrum_matrix(m, n, syn.power_decay(n), BASE_SEED + 7, torch.float32, dev)
    Ai = syn.spectrum_matrix(m, n, syn.power_decay(n), BASE_SEED + 8, torch.float32, dev)
    Ac = torch.complex(Ar, Ai)
    rc = curid.cur_complex(Ac, k, p=10, q=1, seed=5)
    ms_c = timed(lambda: curid.cur_complex(Ac, k, p=10, q=1, seed=5, check=False))
    Acd = Ac.to(torch.complex128)
    Cc, Rc = Acd[:, rc.J[:k].long()], Acd[rc.I[:k].long(), :]
    ec = float(torch.linalg.norm(Acd - Cc @ rc.U @ Rc) / torch.linalg.norm(Acd))
    ms_r = timed(lambda: curid.cur(Ar, k, p=10, q=1, seed=5, check=False))
    res["complex"] = {"workload": f"complex64 A {m}x{n} (real and imaginary parts sigma_j = "
                                  f"j^-2), k = {k}, p = 10, q = 1", "unit": "decompositions/s",
                      "value": 1e3 / ms_c, "ms_per_step": ms_c, "rel_err_fro": ec,
                      "real_path_same_size": {"value": 1e3 / ms_r, "ms_per_step": ms_r}}
    del Ar, Ai, Ac, Acd
    kk, nn = 200, 6000
    g = np.random.default_rng(1)
    S = torch.tensor(np.triu(g.standard_normal((kk, nn))) + np.eye(kk, nn), device=dev)
    J = torch.arange(nn, dtype=torch.int32, device=dev)
    ts = {}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        Sd = S.to(dt)
        ts[name] = {"tikhonov_ms": timed(lambda: curid.interp_tikhonov(Sd, J, kk, 1e-6), 3),
                    "tsvd_ms": timed(lambda: curid.interp_tsvd(Sd, J, kk, 1e-6), 3)}
    res["t_solves"] = {"workload": f"k = {kk}, n = {nn}", **ts}
    torch.cuda.empty_cache()
    return res


def cpu_baseline(args, A, curid):
    """The FP64 oracle on the host cores, one full decomposition of the same
    workload with the Omega the device drew for seed BASE_SEED*1000; returns
    the baseline entry and the oracle's ||A - CUR||_F / ||A||_F."""
    import oracle as O
    l = args.k + args.p
    Om = curid.gaussian(l, args.m, BASE_SEED * 1000, dtype=torch.float32,
                        device=A.device.index).cpu().numpy()
    Ah = A.cpu().numpy()
    t = time.perf_counter()
    o, _ = O.randomized_cur(Ah, Om, args.k, q=args.q)
    dt = time.perf_counter() - t
    err = O.rel_err_fro(Ah.astype(np.float64), o.C, o.U, o.R)
    return ({"value": 1.0 / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
             "sample": f"one full randomized CUR-ID of the same {args.m}x{args.n} float32 A "
                       f"(numpy float64, OpenBLAS threads = all {os.cpu_count()} cores), "
                       f"{dt:.1f} s"}, err)


def run_reference(args, ws, rank, local):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    import oracle as O
    import synthetic as syn
    from oracle.philox import gaussian as philox_gaussian
    dev = "cuda:0" if torch.cuda.is_available() else "cpu"
    A = syn.spectrum_matrix(args.m, args.n, syn.power_decay(min(args.m, args.n)), BASE_SEED,
                            torch.float32, dev).cpu().numpy()
    l = args.k + args.p
    oms = {}

    def step(i):
        seed = BASE_SEED * 1000 + i
        if seed not in oms:
            oms[seed] = philox_gaussian(l, args.m, seed).astype(np.float32)
        O.randomized_cur(A, oms[seed], args.k, q=args.q)

    t0 = time.perf_counter()
    step(0)                                   # one warm-up decomposition
    t_one = time.perf_counter() - t0
    k_steps = max(1, min(args.steps, int(120.0 / max(t_one, 1e-3))))
    for i in range(k_steps):                  # Omega generation outside the timed region
        seed = BASE_SEED * 1000 + 1 + i
        oms[seed] = philox_gaussian(l, args.m, seed).astype(np.float32)
    t0 = time.perf_counter()
    for i in range(k_steps):
        step(1 + i)
    dt = time.perf_counter() - t0
    value = k_steps / dt
    sample = (f"{k_steps} full randomized CUR-ID decompositions of the {args.m}x{args.n} "
              f"workload after 1 warm-up (numpy float64 oracle, {os.cpu_count()} cores)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": k_steps, "warmup": 1, "ms_per_step": dt / k_steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": f"randomized CUR-ID, float32 A {args.m}x{args.n}, k={args.k}, "
                               f"p={args.p}, q={args.q}, Omega {l}x{args.m}",
                   "m": args.m, "n": args.n, "k": args.k, "p": args.p, "q": args.q,
                   "inflight": 1,
                   "l2": "host run", "parallelism": f"{os.cpu_count()} host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.only_form:
        from paper_1412_8447_gb300.build import build
        build()
        dev = torch.device("cuda:0")
        torch.cuda.set_device(dev)
        if args.only_form == "adjoint":
            r = measure_adjoint(dev)
        elif args.only_form == "batched":
            r = measure_batched(dev, nb=256 if args.small else 4096)
        elif args.only_form == "srft":
            r = measure_srft(dev)
        elif args.only_form == "sparse":
            r = measure_sparse(dev)
        elif args.only_form == "extras":
            r = measure_extras(dev)
        elif args.only_form == "c1":
            r = measure_c1(dev)
        else:
            r = (measure_mixed(dev, steps=1, size=8192, q=1, with_f64=False) if args.small
                 else measure_mixed(dev))
        print(json.dumps({"form": args.only_form, **r}))
        return
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
