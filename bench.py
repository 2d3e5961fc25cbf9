#!/usr/bin/env python
"""Benchmark of the state-vector gate-application path on GB300.

Workload (one step): the QFT circuit on n = 30 qubits in complex64
(8 GiB state, larger than L2), 480 gates (30 H, 435 controlled-U1,
15 SWAP), one kernel per gate, from a seeded basis state (sv_init + the
circuit).  value = gate applications per second over all ranks.

Also reported: the dominant kernel's achieved HBM bandwidth against the
measured copy bandwidth (per-launch CUDA events recorded live by the
library's profiler during the timed steps), an end-to-end figure through
the C ABI with the state uploaded from and downloaded to a page-locked host
buffer (sv_host_alloc) every step, the adjoint gradient / forward time ratio on the
hardware-efficient ansatz (n = 20, 10 layers, TFIM, complex64), SM clocks
sampled during the timed region, and the CPU oracle's throughput on a
bounded sample of the same workload.

--impl reference times the CPU oracle alone (the comparison arm).
Multi-GPU: independent replicas (the path does not shard here), one per
rank, weak scaling; no collective on the data path.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QFT n=30 c64 gate-apps/s & % HBM roofline; adjoint grad/forward time ratio"
UNIT = "gate-apps/s"
N_QFT = 30
SEED_QFT = 1001


def job_totals(secs: float, units: float, world: int, device: str = "cpu"):
    """Whole-job timing over ranks: the slowest rank's seconds and the units
    of all ranks (replicas: no data-path collective, only this aggregation).
    Returns (max seconds, total units); world == 1 returns the inputs."""
    if world <= 1:
        return secs, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([secs], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.barrier()
    return float(t.item()), float(u.item())


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes(kernel: str, n: int, amp_bytes: int) -> float:
    """B_alg per launch for the QFT's kernels: 2 * bytes * |A|, A the
    amplitudes the gate changes (H: 2^n, controlled-U1: 2^(n-2),
    SWAP: 2^(n-1)); the basis-state initialisation writes 2^n once."""
    if kernel.startswith("kinit"):
        return 1.0 * amp_bytes * 2 ** n
    if kernel.startswith("kphase"):
        return 2.0 * amp_bytes * 2 ** (n - 2)
    if kernel.startswith("kswap"):
        return 2.0 * amp_bytes * 2 ** (n - 1)
    return 2.0 * amp_bytes * 2 ** n


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if gpu_id:
                cmd += ["-i", gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
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
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.file.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.file.name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_oracle_sample(n: int, n_gates: int, threads: int):
    """Time the CPU oracle (as it stands) on the first `n_gates` gates of the
    QFT at n qubits (complex128 host state).  Returns (gate-apps/s, secs,
    description)."""
    import oracle
    import workloads as W
    oracle.set_threads(threads)
    c = W.qft(n)
    sample = W.Circuit(n, c.gates[:n_gates], 0)
    x = W.random_basis_index(n, SEED_QFT)
    t0 = time.perf_counter()
    oracle.run(sample, None, basis=x)
    dt = time.perf_counter() - t0
    desc = (f"first {n_gates} gates of the n={n} QFT (H + controlled-U1) on a complex128 "
            f"2^{n} host state, {threads} OpenMP threads")
    return n_gates / dt, dt, desc


def qft_reference(n: int, x: int, idx: np.ndarray) -> np.ndarray:
    """Closed form of the QFT of |x> at the amplitude indices idx (the
    circuit's final swaps give the DFT with a + sign):
    exp(2 pi i ((x y) mod 2^n) / 2^n) / 2^(n/2); x y in exact integers."""
    xy = (np.uint64(x) * idx.astype(np.uint64)) & np.uint64((1 << n) - 1)
    return np.exp(2j * np.pi * (xy.astype(np.float64) / float(1 << n))) / 2 ** (n / 2)


def sample_indices(n: int, count: int = 1 << 16, seed: int = 2804) -> np.ndarray:
    import workloads as W
    raw = W.splitmix64_block(seed, 0, count) & np.uint64((1 << n) - 1)
    return np.unique(np.concatenate([raw, np.array([0, (1 << n) - 1], np.uint64)]))


def qft_sample_error(psi: np.ndarray, n: int, x: int) -> dict:
    """Error of a QFT output against its closed form on seeded amplitude
    indices: max |dpsi| and the root-mean-square |dpsi| scaled to the norm
    of the whole difference (sqrt(2^n) * RMS, an estimate of ||dpsi||_2)."""
    idx = sample_indices(n)
    d = np.abs(psi[idx.astype(np.int64)].astype(np.complex128) - qft_reference(n, x, idx))
    return {"max_abs": float(d.max()), "l2_estimate": float(np.sqrt(np.mean(d * d) * 2.0 ** n)),
            "samples": int(idx.size)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    per_step = 3
    vals = []
    for i in range(args.warmup + args.steps):
        v, dt, desc = cpu_oracle_sample(args.n, per_step, threads)
        if i >= args.warmup:
            vals.append(dt)
    total = sum(vals)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"qft n={args.n}, one gate at a time, seeded basis input",
                   "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def host_info() -> dict:
    """Host cores and RAM of the machine the oracle runs on."""
    ram = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemTotal:"):
                    ram = int(line.split()[1]) * 1024
    except OSError:
        pass
    import platform
    return {"cores": os.cpu_count() or 1, "ram_bytes": ram, "machine": platform.machine()}


def oracle_timings() -> dict:
    """The oracle as it stands, timed per configuration on 1 thread and on
    every host core, each on a bounded sample of the configuration's work
    (units per second scaled from the sample; the sample is stated)."""
    import oracle
    import workloads as W
    cores = os.cpu_count() or 1
    out = {"host": host_info()}

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    cases = []
    c0, th0 = W.random_layered(12, 20, 1000)
    cases.append(("C0 random layered n=12 complex128 depth 20", "gate-apps/s",
                  lambda: oracle.run(c0, th0), len(c0.gates), "the whole circuit", len(c0.gates)))
    q = W.qft(30)
    x = W.random_basis_index(30, SEED_QFT)
    q2 = W.Circuit(30, q.gates[:2], 0)
    cases.append(("C1 QFT n=30 (oracle in complex128)", "gate-apps/s",
                  lambda: oracle.run(q2, None, basis=x), 2, "first 2 gates (H, controlled-U1)",
                  len(q.gates)))
    c2, th2 = W.hea(20, 10, 1002)
    H2 = W.tfim(20)
    cases.append(("C2 HEA n=20 L=10 energy", "energies/s",
                  lambda: oracle.energy(c2, th2, H2), 1, "one energy (circuit + TFIM)", 1))
    c3, th3 = W.hea(14, 10, 1003)
    H3 = W.tfim(14)
    cases.append(("C3 batch item: HEA n=14 L=10 energy", "energies/s",
                  lambda: oracle.energy(c3, th3, H3), 1, "one of the 4096 items", 1))
    c4, th4 = W.random_layered(28, 40, 1004)
    c4s = W.Circuit(28, c4.gates[:2], c4.n_params)
    cases.append(("C4 random layered n=28 (oracle in complex128)", "gate-apps/s",
                  lambda: oracle.run(c4s, th4), 2, "first 2 gates (RX, RY)", len(c4.gates)))
    rows = []
    for name, unit, fn, units, sample, total in cases:
        row = {"config": name, "unit": unit, "sample": sample}
        for label, t in (("1_thread", 1), ("all_cores", cores)):
            oracle.set_threads(t)
            secs = timed(fn)
            row[label] = {"threads": t, "seconds": secs, "value": units / secs}
        if unit == "gate-apps/s":
            row["full_circuit_estimate_s_all_cores"] = total / row["all_cores"]["value"]
        rows.append(row)
    oracle.set_threads(cores)
    out["configs"] = rows
    return out


def measured_alu_peaks(torch) -> dict:
    """Library GEMM rates on this GPU as ALU denominators (the driver's
    MEASURED_PEAKS.json has HBM and bf16 only): cuBLAS fp32 SGEMM without
    TF32 (FFMA issue) and fp64 DGEMM, best of a few 8192^3 / 4096^3 runs."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n, reps in (("fp32_ffma_tflops", torch.float32, 8192, 5),
                                  ("fp64_tflops", torch.float64, 4096, 3)):
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            torch.matmul(a, b)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[name] = 2.0 * n ** 3 / best / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["how"] = ("torch.matmul (cuBLAS) fp32 8192^3 with TF32 off and fp64 4096^3, "
                  "best of a few, CUDA events; one FMA = 2 flops")
    return out


def _state_errors(got: np.ndarray, ref: np.ndarray) -> dict:
    d = np.abs(np.asarray(got, np.complex128) - ref)
    g = np.asarray(got, np.complex128)
    return {"max_abs": float(d.max()), "l2": float(np.sqrt(np.sum(d * d))),
            "norm_err": float(abs(1.0 - np.vdot(g, g).real))}


def _rel(g, ref) -> float:
    return float(np.max(np.abs(np.asarray(g) - ref)) / max(float(np.max(np.abs(ref))), 1e-300))


def accuracy(torch, n28_golden: bool = True) -> dict:
    """Each configuration's result against the complex128 oracle (or a closed
    form), on the same seeded inputs: max |dpsi|, ||dpsi||_2 and
    |1 - ||psi||^2| of states; energy and normwise gradient errors."""
    import oracle
    import workloads as W
    from paper_2202_07017_gb300 import Batch, State
    oracle.set_threads(os.cpu_count() or 1)
    out = {}
    # C0: full 4096-amplitude output, complex128
    c0, th0 = W.random_layered(12, 20, 1000)
    st = State(12, "c128").init(0)
    out["C0_layered_n12_c128"] = _state_errors(st.apply_circuit(c0, th0).numpy(),
                                                oracle.run(c0, th0))
    st.close()
    # C2: HEA n=20 L=10, TFIM, complex64: state, energy, sampled gradients
    c2, th2 = W.hea(20, 10, 1002)
    H2 = W.tfim(20)
    ref2 = oracle.run(c2, th2)
    e_ref = oracle.expval(ref2, H2, 20)
    ps = [0, 19, 57, 100, 133, 150, 181, 199]
    g_ref = oracle.grad_param_shift(c2, th2, H2, params=ps)
    row = {}
    for fk in (0, 4):
        st = State(20, "c64").init(0)
        e, g = st.grad(c2, th2, H2, [], fuse_k=fk)
        row[f"fuse_k={fk}"] = dict(_state_errors(st.numpy(), ref2), energy_err=abs(e - e_ref),
                                   grad_rel_err_sampled=_rel(g[ps], g_ref[ps]))
        st.close()
    row["gradient_sample"] = ps
    out["C2_hea_n20_tfim_c64"] = row
    # C3: sampled items of the batch, energies and two items' gradients
    hea14, _ = W.hea(14, 10, 1003)
    mixed = W.mixed_batch(1024, 1003)
    circuits = [hea14] + [m[0] for m in mixed]
    hams = [W.tfim(14)] + [m[2] for m in mixed]
    items = [0] * 4096 + list(range(1, 1025))
    thetas = [W.hea_theta(14, 10, 1003 + i) for i in range(4096)] + [m[1] for m in mixed]
    b = Batch(circuits, hams, items, tune=False)
    e, g = b.run(torch.tensor(np.concatenate(thetas), dtype=torch.float64, device="cuda"))
    e, g = e.cpu().numpy(), g.cpu().numpy()
    b.close()
    offs = np.concatenate([[0], np.cumsum([len(t) for t in thetas])])
    picks = list(range(0, len(items), 64)) + [len(items) - 1]
    e_err = []
    for i in picks:
        c = circuits[items[i]]
        e_err.append(abs(e[i] - oracle.energy(c, thetas[i], hams[items[i]])))
    g_err = []
    for i in (5, 4096 + 3):
        c = circuits[items[i]]
        gr = oracle.grad_param_shift(c, thetas[i], hams[items[i]])
        g_err.append(_rel(g[offs[i]:offs[i + 1]], gr))
    out["C3_batch_c64"] = {"items_checked_energy": len(picks), "max_energy_err": max(e_err),
                           "items_checked_gradient": 2, "max_grad_rel_err": max(g_err)}
    # C4 n=28: fused forward state against the oracle's stored run
    gold = os.path.join(ROOT, "tests", "golden", "layered_n28_d40.npz")
    if n28_golden and os.path.exists(gold):
        z = np.load(gold)
        c4, th4 = W.random_layered(28, 40, 1004)
        st = State(28, "c64").init(0)
        st.apply_circuit(c4, th4, 4)
        idx = torch.from_numpy(z["idx"].astype(np.int64)).to(st.tensor.device)
        got = st.tensor[idx].cpu().numpy().astype(np.complex128)
        e4 = st.expval(W.sum_z(28))
        nrm = st.norm()
        st.close()
        d = np.abs(got - z["amp"])
        out["C4_layered_n28_c64_fused"] = {
            "sampled_amplitudes": int(d.size), "max_abs": float(d.max()),
            "rms_rel": float(np.sqrt(np.mean(d * d) / np.mean(np.abs(z["amp"]) ** 2))),
            "norm_err": abs(1 - nrm), "energy_err": abs(e4 - float(z["energy"]))}
    return out


def adjoint_ratio(torch, reps=3):
    """Hardware-efficient ansatz n = 20, L = 10, TFIM, complex64: forward
    (init + circuit + energy) vs adjoint gradient (H psi + reverse sweep)."""
    import workloads as W
    from paper_2202_07017_gb300 import C64, pack_circuit, pack_pauli, sv_adjoint, sv_alloc
    from paper_2202_07017_gb300 import sv_apply_circuit, sv_expval, sv_free, sv_init
    n, L = 20, 10
    c, theta = W.hea(n, L, 1002)
    pc, pp = pack_circuit(c), pack_pauli(W.tfim(n), n)
    h = sv_alloc(n, C64, torch.cuda.current_stream().cuda_stream)
    try:
        fw, gr = [], []
        for i in range(reps + 1):
            t0 = time.perf_counter()
            sv_init(h, 0)
            sv_apply_circuit(h, pc, theta, 0)
            e = sv_expval(h, pp)
            t1 = time.perf_counter()
            e2, g = sv_adjoint(h, pc, theta, pp)
            t2 = time.perf_counter()
            if i:
                fw.append(t1 - t0)
                gr.append(t2 - t1)
    finally:
        sv_free(h)
    f, gm = float(np.median(fw)), float(np.median(gr))
    fused = _fused_grad_times(torch, c, theta, pc, pp, [], reps)
    return {"workload": "hardware-efficient ansatz n=20 L=10 (200 params), TFIM, complex64",
            "forward_ms": 1e3 * f, "grad_ms": 1e3 * gm, "grad_over_forward": gm / f,
            "energy": e, "fused": {(k[:-2] + "_ms" if k.endswith("_s") else k):
                                   (1e3 * v if k.endswith("_s") else v)
                                   for k, v in fused.items()}}


def _fused_grad_times(torch, c, theta, pc, pp, ck, reps):
    """Forward (init + fused circuit, k = 4 + energy) and forward + gradient
    through sv_grad_fused (fused forward and fused reverse sweep)."""
    from paper_2202_07017_gb300 import (C64, sv_alloc, sv_apply_circuit, sv_expval, sv_free,
                                        sv_grad_fused, sv_init, sv_profile_start,
                                        sv_profile_stop)
    h = sv_alloc(c.n_qubits, C64, torch.cuda.current_stream().cuda_stream)
    try:
        sv_init(h, 0)
        sv_grad_fused(h, pc, theta, pp, ck, 4)  # warm-up (work states, checkpoints)
        fw, fg = [], []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sv_init(h, 0)
            sv_apply_circuit(h, pc, theta, 4)
            sv_expval(h, pp)
            t1 = time.perf_counter()
            sv_init(h, 0)
            sv_profile_start()
            e, g = sv_grad_fused(h, pc, theta, pp, ck, 4)
            t2 = time.perf_counter()
            prof = sv_profile_stop()
            fw.append(t1 - t0)
            fg.append(t2 - t1)
    finally:
        sv_free(h)
    f, t = float(np.median(fw)), float(np.median(fg))
    cnt, ms = prof.get("kfused_adj_c64", (0, 0.0))
    # a reverse pass reads and writes psi and lambda once: 4 * 8 * 2^n bytes
    adj = ({"passes": cnt, "ms": ms, "achieved_gbs": cnt * 32.0 * 2 ** c.n_qubits / (ms / 1e3) / 1e9}
           if cnt else None)
    return {"forward_s": f, "forward_plus_grad_s": t, "grad_over_forward": (t - f) / f,
            "energy": e, "reverse_passes": adj}


def qaoa_maxcut(torch, n=24, p=4, reps=3, n_check=16, check=True):
    """QAOA on MaxCut (3-regular graph, p layers; PAULI "ZZ" cost rotations
    and "X" mixer rotations, 2p parameters), complex64: forward (init +
    circuit + energy) and forward + adjoint gradient, unfused and fused; with
    check (the accuracy leg), the same generator at n_check qubits against
    the oracle's energy and its exact two-term shift rule."""
    import workloads as W
    from paper_2202_07017_gb300 import (C64, pack_circuit, pack_pauli, sv_adjoint, sv_alloc,
                                        sv_apply_circuit, sv_expval, sv_free, sv_init)
    out = {"workload": f"QAOA MaxCut, random 3-regular graph n={n}, p={p} "
                       f"({2 * p} parameters), complex64"}
    for nq, key in ((n, "timed"), (n_check, "check"))[:2 if check else 1]:
        edges = W.random_regular_graph(nq, 3, 4000 + nq)
        c, theta = W.qaoa(nq, edges, p, 4100 + nq)
        H = W.maxcut(edges)
        pc, pp = pack_circuit(c), pack_pauli(H, nq)
        h = sv_alloc(nq, C64, torch.cuda.current_stream().cuda_stream)
        try:
            fw, gr = [], []
            for i in range(reps + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sv_init(h, 0)
                sv_apply_circuit(h, pc, theta, 0)
                e = sv_expval(h, pp)
                t1 = time.perf_counter()
                e2, g = sv_adjoint(h, pc, theta, pp)
                t2 = time.perf_counter()
                if i:
                    fw.append(t1 - t0)
                    gr.append(t2 - t1)
        finally:
            sv_free(h)
        if key == "timed":
            f, gm = float(np.median(fw)), float(np.median(gr))
            fused = _fused_grad_times(torch, c, theta, pc, pp, [], reps)
            out.update({"gates": len(c.gates), "forward_ms": 1e3 * f, "grad_ms": 1e3 * gm,
                        "grad_over_forward": gm / f, "energy": e,
                        "fused": {"forward_ms": 1e3 * fused["forward_s"],
                                  "forward_plus_grad_ms": 1e3 * fused["forward_plus_grad_s"],
                                  "grad_over_forward": fused["grad_over_forward"]}})
        else:
            import oracle
            e_ref = oracle.energy(c, theta, H)
            g_ref = oracle.grad_param_shift(c, theta, H)
            out["error_vs_oracle"] = {"n_qubits": nq, "energy_abs": abs(e2 - e_ref),
                                      "grad_rel_max": _rel(g, g_ref)}
    return out


def followons(torch, n_grover=20, n_trotter=28, steps=10):
    """The scope table's follow-on workloads, timed with CUDA events:
    Grover's search (complex64, n_grover qubits, the optimal iteration count;
    the oracle and the diffusion as n-1-controlled Z gates) unfused and fused,
    with the marked state's probability against its closed form
    sin^2((2k+1) asin 2^(-n/2)); and a first-order Trotter evolution of the
    transverse-field Ising chain (n_trotter qubits, `steps` steps, one Pauli
    rotation pass per term, consecutive diagonal terms merged), with its norm
    error."""
    import math
    import workloads as W
    from paper_2202_07017_gb300 import State
    st_ = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        torch.cuda.synchronize()
        ev[0].record(st_)
        fn()
        ev[1].record(st_)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3

    out = {}
    n = n_grover
    th = math.asin(2.0 ** (-n / 2))
    k = int(math.floor(math.pi / (4 * th)))
    marked = 0xB3C5A5 % (1 << n)
    c = W.grover(n, marked, k)
    g = {"workload": f"Grover search n={n}, {k} iterations ({len(c.gates)} gates, "
                     f"{n - 1}-controlled Z), complex64", "gates": len(c.gates)}
    for fk, mode in ((0, "default"), (4, "dithered")):
        s = State(n, "c64")
        s.set_rounding(mode)
        s.init(0)
        s.apply_circuit(c, None, fk)  # warm-up
        s.init(0)
        secs = timed(lambda: s.apply_circuit(c, None, fk))
        p = s.probabilities(list(range(n)))
        s.close()
        g["fused" if fk else "unfused"] = {
            "seconds": secs, "gate_apps_per_s": len(c.gates) / secs,
            "p_marked_err": abs(float(p[marked]) - math.sin((2 * k + 1) * th) ** 2),
            "norm_err": abs(1.0 - float(np.sum(p))), "rounding": mode}
    out["grover"] = g
    n = n_trotter
    s = State(n, "c64").init(0)
    H = W.tfim(n)
    s.trotter(H, 0.1, 1, 1)  # warm-up
    s.init(0)
    secs = timed(lambda: s.trotter(H, 1.0, steps, 1))
    nrm = s.norm()
    s.close()
    out["trotter"] = {"workload": f"first-order Trotter, TFIM n={n}, {steps} steps "
                                  f"({steps * len(H)} term exponentials), complex64",
                      "seconds": secs, "exponentials_per_s": steps * len(H) / secs,
                      "norm_err": abs(1.0 - nrm)}
    return out


def fused_layered(torch, n=33, depth=40, k=4):
    """Random layered circuit (RX, RY, RZ on every qubit + CZ brick), n = 33
    complex64 (64 GiB), depth 40: fused qubit-block passes for the whole
    circuit, and fused vs one-kernel-per-gate on its first two layers."""
    import workloads as W
    from paper_2202_07017_gb300 import (C64, pack_circuit, sv_alloc, sv_apply_circuit, sv_free,
                                        sv_fusion_plan, sv_init)
    c, theta = W.random_layered(n, depth, 1004)
    pc = pack_circuit(c)
    # the first two layers: 3n rotations each, CZ brick from i = 0 and from i = 1
    layer2 = W.Circuit(n, c.gates[:2 * 3 * n + len(range(0, n - 1, 2)) + len(range(1, n - 1, 2))],
                       c.n_params)
    p2 = pack_circuit(layer2)
    _, _, npass, _ = sv_fusion_plan(pc, theta, C64, k)
    st = torch.cuda.current_stream()
    h = sv_alloc(n, C64, st.cuda_stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        torch.cuda.synchronize()
        ev[0].record(st)
        fn()
        ev[1].record(st)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3

    try:
        sv_init(h, 0)
        sv_apply_circuit(h, p2, theta, k)        # warm-up
        t_full = timed(lambda: sv_apply_circuit(h, pc, theta, k))
        sv_init(h, 0)
        t2_f = timed(lambda: sv_apply_circuit(h, p2, theta, k))
        sv_init(h, 0)
        t2_u = timed(lambda: sv_apply_circuit(h, p2, theta, 0))
    finally:
        sv_free(h)
    pass_bytes = 2 * 8 * 2 ** n
    # arithmetic of the layer programs in rotation form: per circuit layer
    # every qubit's RX RY RZ product is one scaled real rotation on its bit,
    # one FMA per output component (2 per amplitude), and every 4-qubit
    # group applies one complex diagonal (2 FMUL + 2 FFMA per amplitude)
    ffma = float(depth) * (2 * n + 4 * (n / 4)) * 2 ** n
    return {"workload": f"random layered n={n} complex64 depth {depth} ({len(c.gates)} gates), "
                        f"fused register groups of <= {k} qubits",
            "passes": npass, "fused_s": t_full, "gate_apps_per_s": len(c.gates) / t_full,
            "fused_pass_gbs": npass * pass_bytes / t_full / 1e9,
            "alg_fma_ops": ffma, "fma_tops": ffma / t_full / 1e12,
            "first_2_layers": {"gates": len(layer2.gates), "fused_s": t2_f, "unfused_s": t2_u,
                               "speedup": t2_u / t2_f},
            "unfused_full_estimate_s": t2_u * len(c.gates) / len(layer2.gates)}


def qft_c128(torch, n=30, reps=2):
    """The QFT at n = 30 in complex128 (16 GiB state), unfused: gate-apps/s and
    each kernel's algorithmic bandwidth from the library's CUDA events."""
    import workloads as W
    from paper_2202_07017_gb300 import (C128, pack_circuit, sv_alloc, sv_apply_circuit, sv_free,
                                        sv_init, sv_profile_start, sv_profile_stop)
    from paper_2202_07017_gb300 import State
    circ = W.qft(n)
    pc = pack_circuit(circ)
    x = W.random_basis_index(n, SEED_QFT)
    stream = torch.cuda.current_stream()
    st = State(n, "c128")
    h = st.h
    try:
        sv_init(h, x)
        sv_apply_circuit(h, pc, None, 0)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sv_profile_start()
        e0.record(stream)
        for _ in range(reps):
            sv_init(h, x)
            sv_apply_circuit(h, pc, None, 0)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = sv_profile_stop()
        idx = sample_indices(n)
        got = st.tensor[torch.from_numpy(idx.astype(np.int64)).to(st.tensor.device)].cpu().numpy()
        d = np.abs(got - qft_reference(n, x, idx))
        err = {"max_abs": float(d.max()), "l2_estimate": float(np.sqrt(np.mean(d * d) * 2.0 ** n)),
               "norm_err": abs(1.0 - st.norm()), "samples": int(idx.size)}
    finally:
        st.close()
    secs = e0.elapsed_time(e1) / 1e3 / reps
    kernels = {}
    for name, (cnt, ms) in prof.items():
        b = algorithmic_bytes(name, n, 16)
        kernels[name] = {"launches": cnt, "avg_ms": ms / cnt,
                         "achieved_gbs": b * cnt / (ms / 1e3) / 1e9}
        f = fp64_instructions(name, n)
        if f:
            kernels[name]["fp64_instr_per_launch"] = f
            kernels[name]["fp64_tinstr_per_s"] = f * cnt / (ms / 1e3) / 1e12
    return {"workload": f"qft n={n} complex128, unfused, seeded basis input, "
                        f"{len(circ.gates)} gates", "state_bytes": 16 << n,
            "ms_per_step": 1e3 * secs, "gate_apps_per_s": len(circ.gates) / secs,
            "kernels": kernels, "error_vs_closed_form": err}


def fp64_instructions(kernel: str, n: int) -> float:
    """fp64 arithmetic instructions per launch of the complex128 QFT kernels:
    H (a real 2x2) costs 4 multiplies and 4 fused multiply-adds per
    amplitude pair; a controlled U1 phase 2 multiplies and 2 FMAs per
    touched amplitude (2^(n-2)); SWAP and initialisation none."""
    if kernel.startswith("k1q_c128"):
        return 8.0 * 2 ** (n - 1)
    if kernel.startswith("kphase_c128"):
        return 4.0 * 2 ** (n - 2)
    return 0.0


def layered_adjoint(torch, n=28, depth=40):
    """Adjoint gradient of <sum Z_i> for the random layered circuit at n = 28
    (complex64, 3900 gates, 3360 parameters; --adj-n changes n) with forward
    checkpoints every 10 layers: forward (circuit + energy) and forward +
    gradient times, unfused and fused."""
    import workloads as W
    from paper_2202_07017_gb300 import (C64, pack_circuit, pack_pauli, sv_alloc, sv_apply_circuit,
                                        sv_expval, sv_free, sv_grad, sv_init)
    c, theta = W.random_layered(n, depth, 1004)
    pc, pp = pack_circuit(c), pack_pauli(W.sum_z(n), n)
    starts = [i for i, g in enumerate(c.gates) if g.kind == "RX" and g.targets == (0,)]
    ck = [starts[10], starts[20], starts[30]]
    h = sv_alloc(n, C64, torch.cuda.current_stream().cuda_stream)
    try:
        sv_init(h, 0)
        sv_grad(h, pc, theta, pp, ck)  # warm-up (allocates work states and checkpoints)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sv_init(h, 0)
        sv_apply_circuit(h, pc, theta, 0)
        e = sv_expval(h, pp)
        t1 = time.perf_counter()
        sv_init(h, 0)
        e2, g = sv_grad(h, pc, theta, pp, ck)
        t2 = time.perf_counter()
    finally:
        sv_free(h)
    fused = _fused_grad_times(torch, c, theta, pc, pp, ck, 2)
    return {"workload": f"random layered n={n} complex64 depth {depth} ({len(c.gates)} gates, "
                        f"{c.n_params} params), <sum Z>, checkpoints every 10 layers",
            "forward_s": t1 - t0, "forward_plus_grad_s": t2 - t1,
            "grad_over_forward": (t2 - t1 - (t1 - t0)) / (t1 - t0), "energy": e2,
            "fused": fused}


def batch_solves(torch, reps=5, tune=1):
    """4096 parameter sets of the n = 14, L = 10 hardware-efficient ansatz
    plus 1024 mixed ansatz circuits (n 8..16, depth 5..15), TFIM energies and
    adjoint gradients (every gate and term real: the autotuner may pick the
    real-amplitude kernel): one persistent launch per step, replayed from a
    CUDA graph, tile chosen by the autotuner."""
    import workloads as W
    from paper_2202_07017_gb300 import Batch, sv_batch_plan
    hea14, _ = W.hea(14, 10, 1003)
    mixed = W.mixed_batch(1024, 1003)
    circuits = [hea14] + [m[0] for m in mixed]
    hams = [W.tfim(14)] + [m[2] for m in mixed]
    items = [0] * 4096 + list(range(1, 1025))
    theta = np.concatenate([W.hea_theta(14, 10, 1003 + i) for i in range(4096)]
                           + [m[1] for m in mixed])
    t0 = time.perf_counter()
    b = Batch(circuits, hams, items, tune=tune)
    t_create = time.perf_counter() - t0
    th = torch.tensor(theta, dtype=torch.float64, device="cuda")
    e = torch.empty(len(items), dtype=torch.float64, device="cuda")
    g = torch.empty(len(theta), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(3):
        b.run(th, e, g, graph=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(st)
    for _ in range(reps):
        b.run(th, e, g, graph=True)
    ev[1].record(st)
    torch.cuda.synchronize()
    secs = ev[0].elapsed_time(ev[1]) / 1e3 / reps
    # state traffic of the register groups (each group reads and writes the
    # item's states once: psi forward, psi and lambda backward, plus lambda =
    # H psi), against the nominal shared-memory bandwidth of the SMs
    groups = sv_batch_plan(circuits, hams, b.k)
    nq = [c.n_qubits for c in circuits]
    state_bytes = 0.0
    for it in items:
        amp = (4.0 if b.real else 8.0) * 2 ** nq[it]
        state_bytes += amp * (2 * groups[it] + 2 + 4 * groups[it])
    smem_peak = 152 * 128 * 2.07e9 / 1e9  # GB/s: 128 bytes per clock per SM at 2070 MHz
    states = ("real fp32 states (every gate and term real)" if b.real else "complex64")
    out = {"workload": "4096 x HEA n=14 L=10 + 1024 mixed HEA (n 8..16, L 5..15), TFIM, "
                       f"energy + adjoint gradient, {states}, one persistent launch (CUDA graph)",
           "items": len(items), "ms_per_launch": 1e3 * secs, "items_per_s": len(items) / secs,
           "gradients_per_s": len(theta) / secs,
           "tile": {"k": b.k, "threads": b.threads, "blocks": b.blocks, "cluster": b.cluster,
                    "smem_states": b.smem_states, "real_states": b.real},
           "create_and_tune_s": t_create,
           "state_traffic": {"bytes_per_launch": state_bytes,
                             "achieved_gbs": state_bytes / secs / 1e9,
                             "smem_peak_gbs_nominal": smem_peak,
                             "frac": state_bytes / secs / 1e9 / smem_peak}}
    b.close()
    return out


def sampling(torch, h, n, shots=1 << 20):
    """Measurement of all n qubits of the QFT state already in `h`: 2^20 shots
    from seeded uniforms (inverse CDF), and the probabilities of 3 qubits."""
    import workloads as W
    from paper_2202_07017_gb300 import (sv_probabilities, sv_profile_start, sv_profile_stop,
                                        sv_sample)
    u = W.uniform_block(4242, 0, shots)
    q = list(range(n))
    sv_sample(h, q, u[:1024])
    torch.cuda.synchronize()
    sv_profile_start()
    t0 = time.perf_counter()
    sv_sample(h, q, u)
    t1 = time.perf_counter()
    sv_probabilities(h, [0, 1, 2])
    prof = sv_profile_stop()
    cnt, ms = prof.get("kchunk_sums", (1, float("nan")))
    pcnt, pms = prof.get("kprob_slices", (1, float("nan")))
    return {"workload": f"qft n={n} complex64 state, {shots} shots of all qubits "
                        "(inverse CDF, uniforms from the host)",
            "sample_s": t1 - t0, "shots_per_s": shots / (t1 - t0),
            "chunk_sum_gbs": 8 * 2 ** n / (ms / cnt / 1e3) / 1e9,
            "probabilities_gbs": 8 * 2 ** n / (pms / pcnt / 1e3) / 1e9,
            "kernels_ms": {k: v[1] for k, v in prof.items()}}


def reductions(torch, h, n, reps=3):
    """Norm, sum-Z energy (diagonal terms only: one streaming read,
    kdiag_energy) and TFIM energy (its diagonal terms in one streaming read,
    its X terms in three staged passes of kpauli_xbits) of the n = 30 state
    already in `h` (the QFT output): per-kernel times from the library's CUDA
    events, GB/s of each launch of the named kernel (one read of the state,
    8 * 2^n bytes) and the call's time against a single read."""
    import workloads as W
    from paper_2202_07017_gb300 import sv_expval, sv_norm, sv_profile_start, sv_profile_stop
    out = {"workload": f"reductions over the n={n} complex64 QFT state",
           "alg_bytes_per_launch": 8 * 2 ** n}
    peak, _ = hbm_peak()
    cases = (("norm", "knorm", lambda: sv_norm(h)),
             ("energy_sum_z", "kdiag_energy_c64", lambda: sv_expval(h, W.sum_z(n))),
             ("energy_tfim", "kpauli_xbits_c64", lambda: sv_expval(h, W.tfim(n))))
    for name, kern, fn in cases:
        fn()
        sv_profile_start()
        for _ in range(reps):
            v = fn()
        prof = sv_profile_stop()
        cnt, ms = prof.get(kern, (0, float("nan")))
        total_ms = sum(t for _, t in prof.values()) / reps
        per_call = cnt // reps if cnt else 0
        # one read of the state per pass: 8 * 2^n bytes per launch
        out[name] = {"value": v, "kernel": kern, "passes": per_call,
                     "ms_per_call": total_ms,
                     "avg_ms_per_pass": ms / cnt if cnt else None,
                     "pass_gbs": 8 * 2 ** n / (ms / cnt / 1e3) / 1e9 if cnt else None,
                     "pass_frac": 8 * 2 ** n / (ms / cnt / 1e3) / 1e9 / peak if cnt else None,
                     "one_read_frac": 8 * 2 ** n / (total_ms / 1e3) / 1e9 / peak,
                     "kernels_ms": {k: t / reps for k, (c, t) in prof.items()}}
    return out


def gate_table(n, dtype, reps=5):
    """Per-kernel bandwidth for single gates on every kind of bit position:
    H on bit p, controlled-U1 on bits (a, b), SWAP on (a, b).  Algorithmic
    bytes: 2 * amplitude bytes * amplitudes changed."""
    import torch
    from paper_2202_07017_gb300 import State, sv_apply_gate, sv_profile_start, sv_profile_stop
    st = State(n, dtype).init(0)
    amp = 8 if dtype == "c64" else 16
    Hm = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    U1 = np.diag([1, np.exp(0.3j)])
    SW = np.eye(4)[[0, 2, 1, 3]]

    def q(p):
        return n - 1 - p

    cases = [(f"H b{p}", [q(p)], [], Hm, 2 * amp * 2 ** n)
             for p in [0, 1, 2, 3, 4, 5, 8, 12, 16, 20, 24, n - 2, n - 1]]
    cases += [(f"CU1 b{a},{b}", [q(a)], [q(b)], U1, 2 * amp * 2 ** (n - 2))
              for a, b in [(n - 1, 0), (n - 1, 1), (n - 1, 2), (n - 1, 3), (n - 1, 4), (n - 1, 5),
                           (n - 1, 8), (n - 1, 16), (n - 1, n - 2), (15, 0), (15, 14), (1, 0)]]
    cases += [(f"SWAP b{a},{b}", [q(a), q(b)], [], SW, 2 * amp * 2 ** (n - 1))
              for a, b in [(n - 1, 0), (n - 2, 1), (20, 9), (15, 14)]]
    out = []
    for name, t, c, m, balg in cases:
        for _ in range(2):
            sv_apply_gate(st.h, t, c, m)
        torch.cuda.synchronize()
        sv_profile_start()
        for _ in range(reps):
            sv_apply_gate(st.h, t, c, m)
        prof = sv_profile_stop()
        (k, (cnt, ms)), = prof.items()
        out.append({"case": name, "kernel": k, "ms": ms / cnt,
                    "alg_gbs": balg / (ms / cnt / 1e3) / 1e9})
    st.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_QFT)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fused", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adj28", action="store_true")
    ap.add_argument("--no-c128", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--adj-n", type=int, default=28,
                    help="qubits of the layered-circuit adjoint measurement")
    ap.add_argument("--batch-tune", type=int, default=1, choices=[0, 1, 2, 3, 4],
                    help="batch kernel choice: 1 autotune (default), 0 default tile, "
                         "2 clusters, 3 shared-memory states, 4 real states")
    ap.add_argument("--fused-n", type=int, default=33,
                    help="qubits of the fused layered-circuit measurement")
    ap.add_argument("--gate-table", choices=["c64", "c128"],
                    help="print per-kernel bandwidth by bit position and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.gate_table:
        for row in gate_table(args.n, args.gate_table):
            print(json.dumps(row), flush=True)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    import workloads as W
    from paper_2202_07017_gb300 import (C64, pack_circuit, sv_alloc, sv_apply_circuit,
                                        sv_download, sv_free, sv_host_alloc, sv_host_free,
                                        sv_init, sv_launch_count, sv_profile_start,
                                        sv_profile_stop, sv_upload)

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    n = args.n
    circ = W.qft(n)
    pc = pack_circuit(circ)
    n_gates = len(circ.gates)
    x = W.random_basis_index(n, SEED_QFT)
    h = sv_alloc(n, C64, stream.cuda_stream)

    def step():
        sv_init(h, x)
        sv_apply_circuit(h, pc, None, 0)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = str(local)
    clocks = Clocks(gpu_id)
    l0 = sv_launch_count()
    sv_profile_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    prof = sv_profile_stop()
    launches = sv_launch_count() - l0
    clk = clocks.stop()
    secs = e0.elapsed_time(e1) / 1e3
    secs, units = job_totals(secs, n_gates * args.steps, world, "cuda")
    value = units / secs

    # roofline of the dominant kernel, from the live per-launch events
    peak, peak_kind = hbm_peak()
    kernels = {}
    for name, (cnt, ms) in prof.items():
        b = algorithmic_bytes(name, n, 8)
        kernels[name] = {"launches": cnt, "total_ms": ms, "avg_ms": ms / cnt,
                         "alg_bytes_per_launch": b, "achieved_gbs": b * cnt / (ms / 1e3) / 1e9,
                         "share": 0.0}
    tot = sum(k["total_ms"] for k in kernels.values()) or 1.0
    for k in kernels.values():
        k["share"] = k["total_ms"] / tot
    dom = max(kernels, key=lambda k: kernels[k]["total_ms"])
    dk = kernels[dom]
    step_bytes = sum(k["alg_bytes_per_launch"] * k["launches"] for k in kernels.values())
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f).get(dom)
        src = os.path.join(ROOT, "paper_2202_07017_gb300", "csrc", "gate_kernels.cu")
        import hashlib
        if tr and tr.get("source_sha1") == hashlib.sha1(open(src, "rb").read()).hexdigest():
            traffic = tr["dram_bytes_per_launch"]
    except Exception:
        traffic = None
    roofline = {"bound": "hbm", "achieved": dk["achieved_gbs"], "peak": peak, "unit": "GB/s",
                "frac": dk["achieved_gbs"] / peak, "traffic": traffic, "kernel": dom,
                "peak_source": f"{peak_kind} copy bandwidth",
                "frac_of_8000": dk["achieved_gbs"] / 8000.0}

    out = None
    if rank == 0:
        e2e = None
        if not args.no_e2e:
            # page-locked input and output buffers from the library
            # (sv_host_alloc): every step uploads the seeded basis state and
            # downloads the step's result into a separate buffer
            hin = sv_host_alloc(1 << n)
            hout = sv_host_alloc(1 << n)
            try:
                hin[:] = 0
                hin[x] = 1.0
                ts, phases, errs = [], [], []
                for i in range(1 + 4):
                    t0 = time.perf_counter()
                    sv_upload(h, hin)
                    torch.cuda.synchronize()
                    t1 = time.perf_counter()
                    sv_apply_circuit(h, pc, None, 0)
                    torch.cuda.synchronize()
                    t2 = time.perf_counter()
                    sv_download(h, hout)
                    t3 = time.perf_counter()
                    if i:
                        ts.append(t3 - t0)
                        phases.append((t1 - t0, t2 - t1, t3 - t2))
                    errs.append(qft_sample_error(hout, n, x))
            finally:
                sv_host_free(hin)
                sv_host_free(hout)
            ph = np.median(np.array(phases), axis=0)
            e2e = {"value": n_gates / float(np.median(ts)), "unit": UNIT,
                   "h2d_bytes_per_step": 8 << n, "d2h_bytes_per_step": 8 << n,
                   "ms_per_step": 1e3 * float(np.median(ts)),
                   "upload_ms": 1e3 * float(ph[0]), "circuit_ms": 1e3 * float(ph[1]),
                   "download_ms": 1e3 * float(ph[2]),
                   "path": "sv_upload (sv_host_alloc buffer) + sv_apply_circuit + sv_download",
                   "output_check": {"max_abs_err_vs_closed_form": max(e["max_abs"] for e in errs),
                                    "sampled_amplitudes": errs[0]["samples"],
                                    "every_step_from_the_seeded_input": True}}
        meas = sampling(torch, h, n)
        red = reductions(torch, h, n)
        adj = adjoint_ratio(torch)
        qaoa = qaoa_maxcut(torch, check=not args.no_accuracy)
        follow = followons(torch)
        fused = None if args.no_fused else fused_layered(torch, n=args.fused_n)
        batch = None if args.no_batch else batch_solves(torch, tune=args.batch_tune)
        adj28 = None if args.no_adj28 else layered_adjoint(torch, n=args.adj_n)
        c128 = None if args.no_c128 else qft_c128(torch, n=n)
        alu = measured_alu_peaks(torch)
        acc = None if args.no_accuracy else accuracy(torch)
        if acc is not None and e2e is not None:
            acc["C1_qft_n30_c64"] = e2e["output_check"]
        if acc is not None and c128 is not None:
            acc["C1_qft_n30_c128"] = c128["error_vs_closed_form"]
        rooflines = {}
        if fused is not None:
            rooflines["kfused_tma_c64 (random layered n=%d)" % args.fused_n] = {
                "hbm": {"achieved_gbs": fused["fused_pass_gbs"], "peak_gbs": peak,
                        "frac": fused["fused_pass_gbs"] / peak},
                "fma_pipe": {"achieved_tops": fused["fma_tops"],
                             "peak_tops": alu["fp32_ffma_tflops"] / 2,
                             "frac": fused["fma_tops"] / (alu["fp32_ffma_tflops"] / 2)}}
        if adj28 is not None and adj28["fused"].get("reverse_passes"):
            rp = adj28["fused"]["reverse_passes"]
            rooflines["kfused_adj_c64 (layered n=%d)" % args.adj_n] = {
                "bound": "hbm", "achieved_gbs": rp["achieved_gbs"], "peak_gbs": peak,
                "frac": rp["achieved_gbs"] / peak}
        if batch is not None:
            kname = "kbatch_re" if batch["tile"].get("real_states") else "kbatch"
            rooflines[f"{kname} (C3)"] = {"bound": "shared memory (nominal)",
                                          **batch["state_traffic"]}
        for key in ("energy_sum_z", "energy_tfim"):
            r = red[key]
            if r.get("pass_gbs"):
                rooflines[f"{r['kernel']} ({key[7:]} n={n})"] = {
                    "bound": "hbm", "achieved_gbs": r["pass_gbs"], "peak_gbs": peak,
                    "frac": r["pass_frac"], "launches_per_call": r["passes"]}
        if c128 is not None:
            for name, kk in c128["kernels"].items():
                if "fp64_tinstr_per_s" in kk:
                    rooflines[name + " (qft n=30)"] = {
                        "bound": "alu (fp64)", "achieved_tinstr_per_s": kk["fp64_tinstr_per_s"],
                        "peak_tinstr_per_s": alu["fp64_tflops"] / 2,
                        "frac": kk["fp64_tinstr_per_s"] / (alu["fp64_tflops"] / 2),
                        "hbm_frac": kk["achieved_gbs"] / peak}
        cpu = None
        if not args.no_cpu:
            threads = os.cpu_count() or 1
            try:
                v, dt, desc = cpu_oracle_sample(n, 8, threads)
                cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                       "sample": desc, "seconds": dt}
            except MemoryError:
                v, dt, desc = cpu_oracle_sample(28, 8, threads)
                cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                       "sample": desc + " (n=30 did not fit host memory)", "seconds": dt}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"qft n={n} complex64, unfused (one kernel per gate), "
                                   f"seeded basis input, {n_gates} gates",
                       "n_qubits": n, "gates": n_gates, "state_bytes": 8 << n,
                       "l2": (f"inputs larger than L2 ({(8 << n) / 2**30:g} GiB state)"
                              if (8 << n) > 129e6 else
                              f"state of {(8 << n) / 2**20:g} MiB resident in L2 (no flush)"),
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "step_hbm": {"alg_bytes_per_step": step_bytes / args.steps,
                         "achieved_gbs": step_bytes / secs / 1e9,
                         "frac": step_bytes / secs / 1e9 / peak},
            "kernels": kernels,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "adjoint": adj,
            "qaoa": qaoa,
            "followons": follow,
            "fused": fused,
            "batch": batch,
            "adjoint_n28": adj28,
            "qft_c128": c128,
            "measure": meas,
            "reductions": red,
            "accuracy": acc,
            "alu_peaks": alu,
            "rooflines": rooflines,
            "oracle_timings": None if args.no_cpu else oracle_timings(),
        }
    sv_free(h)
    if out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
