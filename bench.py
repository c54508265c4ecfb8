#!/usr/bin/env python3
"""Benchmark of the bit-sliced PCPD sweep on GB300.

Workload (the single-GPU configuration of the headline metric): PCPD on a periodic lattice of
L = 65536 sites, 4096 samples bit-sliced into 32-bit words (128 groups; the "uint64 per site"
of the workload is two such groups), fully occupied start, three runs (d, p) = (0.1, 0.11),
(0.5, 0.15), (0.9, 0.18), Philox seed 1, records at the 100 log-spaced times of a 10^6-MCS
run.  One bench step advances each of the three runs by --mcs-per-step MCS: consecutive
segments of the same 10^6-MCS runs, with the records that fall inside the segment.

Metric: attempted site updates per second (sample x window attempts; S*K per sub-step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): weak scaling by group range -- rank r runs the 4096 samples (128 groups)
[128r, 128r + 128) of one ensemble of 4096*N samples per run (pcpd_params.group0), so the
ranks together reproduce the one-GPU run of that ensemble bit for bit; no data-path
collective (the shards exchange nothing); value = all ranks' attempts / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1301_6082_gb300.replicas import combine, weak_shard  # noqa: E402
from paper_1301_6082_gb300.workloads import SMEM_L65536, batch_instances, log_times, request_stream  # noqa: E402

METRIC = "attempted site updates/s"
# dram__bytes_read.sum + dram__bytes_write.sum of one bench-size launch of the specialised
# sweep (one run advanced 2000 MCS; two 256-thread CTAs per SM, tiles 21848 + 2 x 132 sites,
# tau = 64), 1-pass ncu capture (profiles/pcpd_jit_sweep_L65536_S4096.md)
TRAFFIC_PER_LAUNCH = 38.18e6 + 1738.09e6
# Executed work per (window, group) item of that sweep, from the same capture (d = 1/2):
# widening products = 2 per window + 14 per Philox block x 3.03 blocks (4 FMA-heavy cycles per
# warp instruction), 11.6 other multiply-adds (2 cycles), 29.86 active lanes per warp
# instruction, 1.2% of windows recomputed in tile halos.  Used to predict the FMA-heavy pipe's
# activity from the timed rate, for comparison with ncu's.
EXEC_WIDE_PER_ITEM = 2.0 + 14.0 * 3.03
EXEC_IMAD_PER_ITEM = 11.6
EXEC_ACTIVE_LANES = 29.86
EXEC_HALO = 1.012
UNIT = "attempts/s"


# Integer pipe rates per SM and clock on this GPU (the unit counts: 4 sub-partitions, each
# with a 16-lane ALU pipe and a 16-lane FMA-heavy pipe): 32-bit logic / compare / shift (LOP3
# and kin) take the ALU pipe 2 cycles per warp instruction, 64 lanes per SM and clock; a
# 32x32->64-bit product (Philox's widening multiply, one instruction per product) takes the
# FMA-heavy pipe 4 cycles, 32 products per SM and clock.  The pipe-rate kernels of
# libpcpd_pipes.so measure both (64.0 and 32.0; a pure Philox4x32-10 stream 1.60 blocks =
# 32.0 products per SM and clock), and the bench re-measures the Philox rate on every run.
LOGIC_LANES = 64
WIDE_MUL_LANES = 32
# Shared memory: 32 banks of 4 bytes per SM, one 128-byte wavefront per clock.  A (window,
# group) item of the PCPD reads and writes its three words: 24 bytes.
SMEM_BYTES_PER_CLK = 128
SMEM_BYTES_PER_ITEM = 24


def algorithmic_ops_per_item(t_d: int, t_da: int):
    """Algorithmic integer operations per (window, 32-sample group) item of the method.
    Philox4x32-10: per block 10 rounds x (2 wide multiplies + 2 three-input XORs), times the
    expected number of blocks under the per-item MSB-first early exit; compare: one
    three-input logic op per plane per threshold (2 per expected plane); window logic 11 ops;
    6 shared-memory loads/stores.  Returns (all ops, expected blocks, expected planes,
    wide multiplies, logic-pipe ops)."""
    two32 = 1 << 32

    def p_open(k):  # P(the item is still undecided after k planes)
        cells = set()
        for T in (t_d, t_da):
            if T >= two32 or T == 0:
                continue
            low = T & ((1 << (32 - k)) - 1) if k < 32 else 0
            if low:
                cells.add(T >> (32 - k))
        return 1.0 - (1.0 - len(cells) * 2.0 ** -k) ** 32
    planes = sum(p_open(k) for k in range(32))
    blocks = 1.0 + sum(p_open(k) for k in (3, 7, 11, 15, 19, 23, 27, 31))
    mul = 20.0 * blocks
    logic = 20.0 * blocks + 2.0 * planes + 11.0
    return mul + logic + 6.0, blocks, planes, mul, logic


def pipe_roofline(items_per_s: float, mul_per_item: float, logic_per_item: float, sm_count: int,
                  mhz: float) -> dict:
    """Fractions of the two integer pipes the work needs; the larger one binds."""
    peak_mul = sm_count * WIDE_MUL_LANES * mhz * 1e6
    peak_logic = sm_count * LOGIC_LANES * mhz * 1e6
    f_mul = items_per_s * mul_per_item / peak_mul
    f_logic = items_per_s * logic_per_item / peak_logic
    if f_mul >= f_logic:
        return {"achieved": items_per_s * mul_per_item / 1e12, "peak": peak_mul / 1e12,
                "unit": "T wide-multiply ops/s", "frac": f_mul, "binding_pipe": "32x32->64 multiply (FMA pipe)",
                "frac_logic_pipe": f_logic}
    return {"achieved": items_per_s * logic_per_item / 1e12, "peak": peak_logic / 1e12,
            "unit": "T logic ops/s", "frac": f_logic, "binding_pipe": "32-bit logic (ALU pipe)",
            "frac_wide_multiply_pipe": f_mul}


def measured_peak(key: str, default: float) -> float:
    """A figure from MEASURED_PEAKS.json (the measured copy bandwidth, clocks), else default."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))[key])
    except Exception:
        return default


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"pcpd_bench_clocks_rank{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def host_cores() -> int:
    """Cores this process may run on (its CPU affinity), else the machine's count."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_cpu_sample(budget_groups: int | None = None, substeps: int = 300):
    """The oracle as it stands, on a bounded sample of the workload: one 32-sample group per
    host core the process may run on (at least 16 groups) of the L=65536 lattice at (d,p) =
    (0.5, 0.15), `substeps` sub-steps from the full start, one oracle thread per core (the
    oracle splits its work by group)."""
    from oracle import oracle as O
    L = SMEM_L65536["L"]
    avail = host_cores()
    groups = budget_groups or max(16, avail)
    S = 32 * groups
    d, p = 0.5, 0.15
    cores = min(avail, groups)
    st = O.init_state(L, S, O.MODE_FULL, 1)
    t0 = time.perf_counter()
    O.run(st, p, d, 1, 0, substeps, threads=cores)
    dt = time.perf_counter() - t0
    attempts = S * (L // 3) * substeps
    return {"value": attempts / dt, "unit": UNIT, "cores": cores, "host_cores": avail, "kind": "oracle",
            "value_per_core": attempts / dt / cores,
            "sample": f"{groups} groups ({S} samples) of L={L}, d=0.5 p=0.15, {substeps} sub-steps "
                      f"from full ({attempts:.3e} attempts, {dt:.1f} s, {cores} threads on {avail} cores)"}


def run_rs_sample(samples: int = 256, mcs: int = 40):
    """Alg. 1 (random-sequential, the paper's "conventional" dynamics) as the oracle runs it,
    on L = 65536 with `samples` samples for `mcs` MCS from the full start: the analogue of the
    paper's simple-CPU-program figure."""
    from oracle import oracle as O
    L = SMEM_L65536["L"]
    cores = min(host_cores(), samples)
    st = O.init_state(L, samples, O.MODE_FULL, 1)
    t0 = time.perf_counter()
    O.rs_run(st, 0.15, 0.5, 1, 0, mcs * L, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": samples * L * mcs / dt, "unit": UNIT, "cores": cores,
            "sample": f"Alg. 1 on L={L}, {samples} samples, {mcs} MCS ({dt:.1f} s)"}


PAPER_CONTEXT = {
    "note": "the paper's own numbers (Sec. 5.2), other hardware and schedule: context only",
    "gpu_moves_per_s": 8.0e10, "gpu": "NVIDIA GTX 580 (Fermi), OpenCL via CUDA 4.0, d = 1/2, 32-bit multispin",
    "gpu_over_simple_cpu": 4000, "gpu_over_same_algorithm_on_cpu": 130,
    "cpu": "Intel Xeon E5620 2.4 GHz / Core 2 Duo E8400 3.0 GHz, gcc 4.1.2 -O2",
}


def batch_leg(pcpd, mcs_div: int = 100):
    """The 512-instance heterogeneous mix (L log-uniform 2^10..2^18, 64/256/1024 samples,
    d in {.1,...,.9}, p in [.05,.25], MCS log-uniform 1e3..1e5, full or half start, seeds
    1000+i), with every MCS count divided by mcs_div (declared scale-down; the full mix is
    ~2.3e14 attempts).  Plain = one engine launch per instance, back to back on one stream;
    batched = pcpd_batch_run (one persistent launch per 128 instances).  Same results."""
    import numpy as np
    import torch
    mix = batch_instances(512, seed=1)
    for m in mix:
        m["mcs_run"] = max(1, m["mcs"] // mcs_div)
    attempts = sum(m["S"] * (m["L"] // 3) * pcpd.substep_of_time(m["L"], m["mcs_run"]) for m in mix)
    stream = torch.cuda.Stream()
    # plain
    # both sides run the generic engine (a batch shares one kernel across thresholds)
    sims = [pcpd.Pcpd(m["L"], m["S"], m["p"], m["d"], seed=m["seed"], init=m["init"], stream=stream, jit=-1)
            for m in mix]
    torch.cuda.synchronize()
    l0 = pcpd.kernel_launches()
    t0 = time.perf_counter()
    for s_, m in zip(sims, mix):
        s_.run(m["mcs_run"], [m["mcs_run"]])
    stream.synchronize()
    t_plain = time.perf_counter() - t0
    plain_launches = pcpd.kernel_launches() - l0
    plain_counts = [s_.counts()[-1] for s_ in sims]
    for s_ in sims:
        s_.close()
    # batched
    b = pcpd.Batch(stream=stream)
    for m in mix:
        b.add(m["L"], m["S"], m["p"], m["d"], m["seed"], m["mcs_run"], [m["mcs_run"]], init=m["init"])
    torch.cuda.synchronize()
    l0 = pcpd.kernel_launches()
    t0 = time.perf_counter()
    b.run()
    t_batch = time.perf_counter() - t0
    batch_launches = pcpd.kernel_launches() - l0
    same = all(int(b.counts(i)[-1]) == int(c) for i, c in enumerate(plain_counts))
    b.close()
    # the batched rate against the same multiply-pipe roofline as the headline sweep: each
    # member's algorithmic widening products (its expected Philox blocks x 20 per item)
    products = 0.0
    for m in mix:
        td, tda = pcpd.thresholds(m["p"], m["d"])
        items = m["S"] // 32 * (m["L"] // 3) * pcpd.substep_of_time(m["L"], m["mcs_run"])
        products += items * algorithmic_ops_per_item(td, tda)[3]
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peak = props.multi_processor_count * WIDE_MUL_LANES * measured_peak("sm_max_mhz", 2070.0) * 1e6
    return {"workload": "512-instance mix, MCS/%d" % mcs_div, "attempts": attempts,
            "batched": attempts / t_batch, "plain": attempts / t_plain, "unit": UNIT,
            "speedup": t_plain / t_batch, "batched_launches": batch_launches, "plain_launches": plain_launches,
            "results_identical": bool(same), "frac": round(products / t_batch / peak, 4),
            "frac_plain": round(products / t_plain / peak, 4),
            "frac_note": "algorithmic widening products of every member / wall time / the headline sweep's peak"}


def sweep_batch_leg(pcpd, mcs: int = 300):
    """A near-critical sweep as one batch (Sec. 5.3): d = 1/2, p in {0.12, 0.13, 0.14, 0.15},
    4 seeds each, L = 65536, 1024 samples, full start, `mcs` MCS.  The members of one p share
    their thresholds, so their launches can run the engine compiled for them (timed after the
    compiles, which a process pays once per pair) against the generic kernel.  Same records."""
    import torch
    ps, seeds, L, S = (0.12, 0.13, 0.14, 0.15), (1, 2, 3, 4), 65536, 1024
    times = [mcs]
    out = {}
    counts = {}
    for mode in (1, -1, 1):   # the first pass compiles; the second and third are timed
        b = pcpd.Batch()
        b.set_jit(mode)
        for p in ps:
            for sd in seeds:
                b.add(L, S, p, 0.5, sd, mcs, times)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run()
        dt = time.perf_counter() - t0
        attempts = len(ps) * len(seeds) * S * (L // 3) * pcpd.substep_of_time(L, mcs)
        counts[mode] = [int(b.counts(i)[-1]) for i in range(len(ps) * len(seeds))]
        out["specialised" if mode > 0 else "generic"] = {"value": attempts / dt, "jit_launches": b.jit_launches}
        b.close()
    return {"workload": "sweep batch: d=0.5, p in %s x %d seeds, L=%d, %d samples, %d MCS" % (ps, len(seeds), L, S, mcs),
            "unit": UNIT, **out, "speedup": out["specialised"]["value"] / out["generic"]["value"],
            "results_identical": counts[1] == counts[-1]}


def stream_leg(pcpd, substeps: int = 2048):
    """The HBM-streamed workload: L = 2^22 sites, 1024 samples, d=0.5, p=0.15, full start,
    seed 1 (the lattice, 2 x 512 MiB, is far larger than shared memory and L2, so every
    epoch of tau sub-steps streams each tile in with its halo and its core back out).
    Times `substeps` sub-steps after one warm-up epoch; HBM bytes are the algorithmic tile
    traffic (tile with halo read + core written, per epoch)."""
    import torch
    L, S = 1 << 22, 1024
    stream = torch.cuda.Stream()
    sim = pcpd.Pcpd(L, S, 0.15, 0.5, seed=1, stream=stream)
    sim.run_substeps(256)
    sim.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.run_substeps(substeps)
    ev1.record(stream)
    sim.sync()
    ms = ev0.elapsed_time(ev1)
    plan = sim.plan()
    epochs = -(-substeps // plan["tau"])
    G = S // 32
    tile_bytes = G * (L + plan["n_seg"] * 2 * plan["halo"]) * 4 + G * L * 4
    hbm = tile_bytes * epochs / (ms / 1e3) / 1e9
    sim.close()
    return {"workload": "L=2^22, 1024 samples, d=0.5, p=0.15, %d sub-steps" % substeps,
            "value": S * (L // 3) * substeps / (ms / 1e3), "unit": UNIT, "plan": plan,
            "hbm_gbs_algorithmic": hbm, "hbm_frac_of_measured_copy": hbm / measured_peak("hbm_gbs", 6787.2)}


def tuple_leg(pcpd, mcs: int = 500):
    """The n-tuple processes (TCPD n = 3, QCPD n = 4; windows of n+1 sites) on the headline
    lattice: L = 65536, 4096 samples, full start, d = 0.5, p = 0.15, seed 1; `mcs` MCS timed
    after 5 MCS of warm-up, through the same engine (specialised at run time)."""
    import torch
    out = []
    for n in (3, 4):
        L, S = 65536, 4096
        stream = torch.cuda.Stream()
        sim = pcpd.Pcpd(L, S, 0.15, 0.5, seed=1, stream=stream, tuple_n=n)
        sim.run(5)
        sim.sync()
        n0 = sim.substep
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sim.run(mcs, [5 + mcs])
        ev1.record(stream)
        sim.sync()
        ms = ev0.elapsed_time(ev1)
        K = L // (n + 1)
        items = (S // 32) * K * (sim.substep - n0)
        td, tda = pcpd.thresholds(0.15, 0.5)
        _, blocks, _, mul, logic = algorithmic_ops_per_item(td, tda)
        logic += 2.0 * (n - 2) + 3.0 * (n - 2)          # wider tuple test and updates
        rate = items * 32 / (ms / 1e3)
        out.append({"tuple": n, "L": L, "samples": S, "mcs": mcs, "value": rate, "unit": UNIT, "ms": ms,
                    "rho_end": float(sim.density()[-1]), "plan": sim.plan(),
                    "roofline": {"bound": "alu", **pipe_roofline(items / (ms / 1e3), mul, logic,
                                                                  torch.cuda.get_device_properties(
                                                                      torch.cuda.current_device()).multi_processor_count,
                                                                  2070.0)}})
        sim.close()
    return {"workload": "TCPD / QCPD, L=65536, 4096 samples, d=0.5, p=0.15, %d MCS" % mcs, "runs": out}


def paper_ops_per_step_thread(m: int, n_dec: int):
    """Algorithmic integer operations per (step, thread) of the paper's scheme: Philox4x32-10
    blocks ((m + n_dec + 2)/4 mask blocks, as four steps share whole blocks, and 1/128 of a
    local-site block) at 20 wide multiplies + 20 three-input XORs each; 2 logic ops per
    diffusion plane, 1 per decorrelation word, 2 for the broadcast compare, 12 for the bond
    logic of Alg. 2; 8 shared-memory loads/stores.  One (step, thread) = 32 attempts.
    Returns (all ops, blocks, wide multiplies, logic-pipe ops)."""
    blocks = (m + n_dec + 2) / 4.0 + 1.0 / 128.0
    mul = 20.0 * blocks
    logic = 20.0 * blocks + 2.0 * m + n_dec + 2.0 + 12.0
    return mul + logic + 8.0, blocks, mul, logic


def paper_leg(pcpd, mcs: int = 1000, systems: int = 3648):
    """The paper's own scheme (Sec. 3-4, Alg. 2) at the layout it reports: rings of
    L = 65536 sites (S_w = 64 threads x n_loc = 32 words, and S_w = 32 x 64), d = 1/2
    (m = 1 plane), n_dec = 2 decorrelation words, p = 0.15, full start, `systems` systems
    (3648 = 152 SMs x 24 resident systems: one full wave), 20 log-spaced records; `mcs` MCS
    timed after 1 MCS of warm-up."""
    import torch
    out = []
    m, n_dec = 1, 2
    ops, blocks, mul, logic = paper_ops_per_step_thread(m, n_dec)
    sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    for n_loc, S_w in ((32, 64), (64, 32)):
        L = 32 * n_loc * S_w
        stream = torch.cuda.Stream()
        h = pcpd.PaperScheme(n_loc, S_w, systems, 0.15, 0.5, m, n_dec, seed=1, stream=stream)
        h.run(n_loc)
        h.sync()
        recs = sorted({n_loc * int(t) for t in log_times(mcs + 1, 20) if t > 1})
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        h.run(mcs * n_loc, recs)
        ev1.record(stream)
        h.sync()
        ms = ev0.elapsed_time(ev1)
        rate = systems * L * mcs / (ms / 1e3)
        step_threads = rate / 32.0
        out.append({"n_loc": n_loc, "S_w": S_w, "L": L, "systems": systems, "mcs": mcs,
                    "value": rate, "unit": UNIT, "ms": ms, "plan": h.plan(),
                    "rho_end": float(h.density()[-1]),
                    "roofline": {"bound": "alu", **pipe_roofline(step_threads, mul, logic, sm_count, 2070.0),
                                 "ops_per_step_thread": ops, "philox_blocks_per_step_thread": blocks}})
        h.close()
    # rate against the workgroup size at the same L (the paper's performance-vs-S_w study,
    # Sec. 5.2): S_w = 32 .. 512 threads per system, n_loc = 65536 / (32 S_w), 200 MCS each
    by_sw = []
    for S_w in (32, 64, 128, 256, 512):
        n_loc = 65536 // (32 * S_w)
        stream = torch.cuda.Stream()
        h = pcpd.PaperScheme(n_loc, S_w, systems, 0.15, 0.5, m, n_dec, seed=1, stream=stream)
        h.run(n_loc)
        h.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        h.run(200 * n_loc)
        ev1.record(stream)
        h.sync()
        ms = ev0.elapsed_time(ev1)
        by_sw.append({"S_w": S_w, "n_loc": n_loc, "value": systems * 65536 * 200 / (ms / 1e3),
                      "plan": h.plan()})
        h.close()
    return {"workload": "paper scheme, L=65536, %d systems, d=0.5 (m=1), n_dec=2, p=0.15, %d MCS"
            % (systems, mcs), "runs": out, "by_workgroup_size": by_sw,
            "note": "a different Markov chain from the main path (shared local site, correlated "
                    "annihilation draws); same unit as the paper's moves/s"}


def serving_run(pcpd, reqs, seconds: float):
    """Submit `reqs` at their Poisson arrival times to a fresh server; wait for all of them.
    Returns (throughput in attempts/s over the wall time, p50, p99 latency, stats)."""
    import numpy as np
    sv = pcpd.Server(hbm_budget_bytes=96 << 30, max_active=128, chunk_attempts=4 << 30)
    ids = []
    t0 = time.perf_counter()
    for r in reqs:
        wait = r["arrival"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ids.append(sv.submit(r["L"], r["S"], r["p"], r["d"], r["seed"], r["mcs"], [r["mcs"]], init=r["init"]))
    sv.wait_idle()
    wall = time.perf_counter() - t0
    lat = np.array([sv.result(i)[2] for i in ids])
    st = sv.stats()
    sv.stop()
    return st["attempts"] / wall, float(np.percentile(lat, 50)), float(np.percentile(lat, 99)), st, wall


def serving_leg(pcpd, seconds: float = 8.0, rate_hz: float = 200.0, fractions=(0.5, 0.75, 1.0, 1.25)):
    """Poisson request stream (200 req/s; L log-uniform 2^10..2^20, 64..4096 samples,
    p in [.05,.25], d in [.1,.9], MCS log-uniform 1e3..1e5) for `seconds` instead of 60 s, with
    every MCS count scaled down (declared: as specified the stream offers ~7.6e14 attempts/s,
    hundreds of times one GPU's capacity).  First the capacity: the same requests (MCS x 1/600)
    all submitted at once, attempts/s until the last finishes.  Then the load curve: the stream
    with its MCS scaled so that it offers each fraction of that capacity; throughput and p50/p99
    latency from submission to result at each point."""
    base_scale = 1 / 600
    base = request_stream(rate_hz, seconds, seed=1, mcs_scale=base_scale)
    offered_base = sum(r["S"] * (r["L"] // 3) * pcpd.substep_of_time(r["L"], r["mcs"]) for r in base) / seconds
    burst = [dict(r, arrival=0.0) for r in base]
    capacity, _, _, _, _ = serving_run(pcpd, burst, seconds)
    curve = []
    for f in fractions:
        scale = base_scale * f * capacity / offered_base
        reqs = request_stream(rate_hz, seconds, seed=1, mcs_scale=scale)
        offered = sum(r["S"] * (r["L"] // 3) * pcpd.substep_of_time(r["L"], r["mcs"]) for r in reqs) / seconds
        thr, p50, p99, st, wall = serving_run(pcpd, reqs, seconds)
        curve.append({"load": f, "offered": offered, "throughput": thr, "p50_latency_s": p50, "p99_latency_s": p99,
                      "requests": len(reqs), "completed": int(st["completed"]), "rounds": int(st["rounds"]),
                      "wall_s": wall, "mcs_scale": scale})
    at = min(curve, key=lambda c: abs(c["load"] - 0.75))
    return {"workload": "Poisson %g req/s for %g s, MCS scaled to a fraction of capacity" % (rate_hz, seconds),
            "unit": UNIT, "capacity": capacity, "curve": curve,
            "throughput": at["throughput"], "p50_latency_s": at["p50_latency_s"], "p99_latency_s": at["p99_latency_s"],
            "at_load": at["load"]}


def reference_arm(args, world, rank):
    """The oracle timed on the host cores, one bounded sample of the workload per step."""
    if rank != 0:
        return 0
    groups, subs = host_cores(), 60   # one 32-sample group per host core, all cores busy
    res = None
    times = []
    for i in range(args.warmup + args.steps):
        r = run_cpu_sample(groups, subs)
        if i >= args.warmup:
            times.append(r)
        res = r
    vals = [r["value"] for r in times]
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * (32 * groups * (SMEM_L65536["L"] // 3) * subs) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": SMEM_L65536["name"], "L": SMEM_L65536["L"], "samples": SMEM_L65536["S"],
                       "note": "each step: the CPU oracle on a bounded sample of the workload"},
            "cpu_baseline": {"kind": "oracle", "cores": res["cores"], "host_cores": res["host_cores"],
                             "sample": res["sample"], "value": value,
                             "unit": UNIT, "value_per_core": value / res["cores"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def compact(d, keys):
    """The named entries of a leg's result (None stays None)."""
    return None if d is None else {k: d[k] for k in keys if k in d}


def compact_roofline(r):
    """The roofline entries the headline line carries; the notes go to the detail line."""
    keep = ("bound", "achieved", "peak", "unit", "frac", "traffic", "frac_logic_pipe",
            "frac_of_issue_slots", "frac_smem", "peak_measured", "fmaheavy_active_pred")
    out = {k: r[k] for k in keep if k in r}
    for k in ("achieved", "peak", "frac", "frac_logic_pipe", "frac_of_issue_slots", "frac_smem", "peak_measured",
              "fmaheavy_active_pred"):
        if isinstance(out.get(k), float):
            out[k] = round(out[k], 4)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mcs-per-step", type=int, default=2000)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    ap.add_argument("--no-tuples", action="store_true")
    ap.add_argument("--paper-only", action="store_true",
                    help="run only the paper-scheme leg (for profiling) and print its JSON")
    ap.add_argument("--paper-mcs", type=int, default=1000)
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the 512-instance batch leg (for profiling) and print its JSON")
    ap.add_argument("--batch-mcs-div", type=int, default=100,
                    help="divide every MCS count of the 512-instance mix by this (1 = the mix as specified)")
    ap.add_argument("--stream-only", action="store_true",
                    help="run only the HBM-streamed leg (for profiling) and print its JSON")
    ap.add_argument("--stream-substeps", type=int, default=2048)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world, rank, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import numpy as np
    import torch
    from paper_1301_6082_gb300 import build as B
    B.build()
    from paper_1301_6082_gb300 import pcpd

    torch.cuda.set_device(local)
    if args.paper_only:
        print(json.dumps({"paper_scheme": paper_leg(pcpd, mcs=args.paper_mcs)}), flush=True)
        return 0
    if args.batch_only:
        print(json.dumps({"batch": batch_leg(pcpd, mcs_div=max(1, args.batch_mcs_div))}), flush=True)
        return 0
    if args.stream_only:
        print(json.dumps({"streamed": stream_leg(pcpd, substeps=args.stream_substeps)}), flush=True)
        return 0
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    W = SMEM_L65536
    L, S = W["L"], W["S"]
    K_win = L // 3
    runs = W["runs"]
    rec_all = log_times(W["mcs"], W["n_rec"])
    # the three runs are independent: one stream each, so one launch's tail overlaps the next
    streams = [torch.cuda.Stream() for _ in runs]
    main_stream = torch.cuda.Stream()
    g0, _ = weak_shard(S // 32, rank)   # this rank's groups of the 4096*world-sample ensemble
    sims = []
    for i, (d, p) in enumerate(runs):
        sims.append(pcpd.Pcpd(L, S, p, d, seed=W["seed"], stream=streams[i], group0=g0))
    ops_item = []
    for d, p in runs:
        td, tda = pcpd.thresholds(p, d)
        ops_item.append(algorithmic_ops_per_item(td, tda))

    mcs = args.mcs_per_step

    def step(sim_list, t0):
        recs = [t for t in rec_all if t0 < t <= t0 + mcs]
        for s in sim_list:
            s.run(mcs, recs)

    t_now = 0
    for _ in range(args.warmup):
        step(sims, t_now)
        t_now += mcs
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sub0 = [s.substep for s in sims]
    launches0 = pcpd.kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(main_stream)
    for st in streams:
        st.wait_event(ev0)
    for _ in range(args.steps):
        step(sims, t_now)
        t_now += mcs
    for st in streams:            # the end event waits for every run's stream
        done = torch.cuda.Event()
        done.record(st)
        main_stream.wait_event(done)
    ev1.record(main_stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = pcpd.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    subs = [s.substep - a for s, a in zip(sims, sub0)]
    attempts = sum(S * K_win * n for n in subs)
    alg_ops = sum(S // 32 * K_win * n * o[0] for n, o in zip(subs, ops_item))   # this rank
    (attempts_all,), (ms_max,) = combine(dist, [attempts], [ms], device="cuda")
    value = attempts_all / (ms_max / 1e3)

    # roofline of the dominant kernel (the tile sweep): the binding integer pipe
    props = torch.cuda.get_device_properties(local)
    sm_count = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    items = [S // 32 * K_win * n for n in subs]            # (window, group) items, this rank
    items_s = sum(items) / (ms / 1e3)
    mul_item = sum(i * o[3] for i, o in zip(items, ops_item)) / sum(items)
    logic_item = sum(i * o[4] for i, o in zip(items, ops_item)) / sum(items)
    plan0 = sims[0].plan()
    pipe_rates = None
    try:   # the measured peak beside the derived one: a pure Philox stream on this GPU
        from paper_1301_6082_gb300 import pipes as PR
        B.build_pipes()
        pipe_rates = {op: round(PR.rate(op)[0], 2) for op in ("philox", "imad_wide", "lop3")}
        pipe_rates["philox_products"] = round(20.0 * pipe_rates["philox"], 2)
    except Exception as exc:   # reported, not fatal: the derived peak stands
        pipe_rates = {"error": str(exc)[:200]}
    kname = "pcpd_jit_sweep (engine compiled for the run's thresholds)" if plan0.get("jit") else "k_sweep_persistent"
    issue_peak = sm_count * 4 * 32 * sm_max_mhz * 1e6 / 1e12   # T lane-ops/s, all pipes together
    roofline = {"bound": "alu", **pipe_roofline(items_s, mul_item, logic_item, sm_count, sm_max_mhz),
                "traffic": TRAFFIC_PER_LAUNCH if plan0.get("jit") else None,
                "kernel": f"{kname}; tiles {plan0['core']}+2x{plan0['halo']} sites, tau={plan0['tau']}",
                "peak_note": f"{sm_count} SMs x {WIDE_MUL_LANES} wide-multiply / {LOGIC_LANES} logic lanes x "
                             f"{sm_max_mhz:.0f} MHz (derived from the unit counts; lane rates checked by a microbenchmark of independent dependency chains)",
                "achieved_note": "algorithmic wide multiplies of all sweep launches in the timed region "
                                 "(the three runs on their own streams) / the region's CUDA-event duration",
                "wide_multiplies_per_item": round(mul_item, 2), "logic_ops_per_item": round(logic_item, 2),
                "expected_philox_blocks_per_item": [round(o[1], 3) for o in ops_item],
                "frac_of_issue_slots": (alg_ops / (ms / 1e3)) / 1e12 / issue_peak,
                "frac_smem": items_s * SMEM_BYTES_PER_ITEM / (sm_count * SMEM_BYTES_PER_CLK * sm_max_mhz * 1e6),
                "measured_lanes_per_sm_clock": pipe_rates,
                "fmaheavy_active_pred": items_s * (EXEC_WIDE_PER_ITEM * 4 + EXEC_IMAD_PER_ITEM * 2) / EXEC_ACTIVE_LANES
                * EXEC_HALO / (4 * sm_count * sm_max_mhz * 1e6),
                "peak_measured": (pipe_rates.get("philox_products", 0) * sm_count * sm_max_mhz * 1e6 / 1e12
                                  if "philox_products" in pipe_rates else None)}

    # end to end through the public API with host buffers (pinned), host<->device in the region:
    # each run on its own stream, so one run's copies overlap another run's sweep
    e2e = None
    if args.e2e_steps > 0:
        host = [torch.empty((S // 32, L), dtype=torch.int32, pin_memory=True) for _ in sims]
        streams = [torch.cuda.Stream() for _ in sims]
        esims = [pcpd.Pcpd(L, S, p, d, seed=W["seed"], stream=st, group0=g0)
                 for (d, p), st in zip(runs, streams)]
        for es, s, hb in zip(esims, sims, host):
            arr = hb.numpy().view(np.uint32)
            s.lattice(out=arr)
            es.set_lattice(arr, s.substep)        # continue where the timed runs stopped
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        att_e2e, h2d, d2h = 0, 0, 0
        for _ in range(args.e2e_steps):
            n0s = []
            for es, hb in zip(esims, host):
                arr = hb.numpy().view(np.uint32)
                es.set_lattice(arr, es.substep, wait=False)
                h2d += arr.nbytes
                n0s.append(es.substep)
                recs = [t for t in rec_all if es.time_mcs < t <= es.time_mcs + mcs]
                es.run(mcs, recs)
            for es, hb in zip(esims, host):
                es.lattice(out=hb.numpy().view(np.uint32), wait=False)
                d2h += hb.numel() * 4
            for es, n0 in zip(esims, n0s):
                es.sync()
                rho = es.density()
                d2h += rho.nbytes
                att_e2e += S * K_win * (es.substep - n0)
        dt = time.perf_counter() - t0
        for es in esims:
            es.close()
        e2e_val = att_e2e / dt
        if dist:
            (att_all,), (dt_max,) = combine(dist, [att_e2e], [dt], device="cuda")
            e2e_val = att_all / dt_max
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d // args.e2e_steps,
               "d2h_bytes_per_step": d2h // args.e2e_steps,
               "note": "per run per step, each run on its own stream: pcpd_set_lattice_async from pinned host "
                       "memory, pcpd_run, pcpd_get_lattice_async into pinned memory, pcpd_sync, pcpd_density"}

    for s in sims:
        s.close()
    sims = []
    batch = batch_leg(pcpd) if not args.no_batch else None
    sweep_batch = sweep_batch_leg(pcpd) if not args.no_batch else None
    serving = serving_leg(pcpd) if not args.no_serve else None
    streamed = stream_leg(pcpd, substeps=args.stream_substeps) if not args.no_stream else None
    paper = paper_leg(pcpd, mcs=args.paper_mcs) if not args.no_paper else None
    tuples = tuple_leg(pcpd) if not args.no_tuples else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_sample()
        cpu["alg1_random_sequential"] = run_rs_sample()

    if rank == 0:
        # every leg in full on an earlier line; the headline line (printed last) stays short
        detail = {"roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "batch": batch,
                  "sweep_batch": sweep_batch, "serving": serving,
                  "streamed": streamed, "paper_scheme": paper, "tuples": tuples,
                  "paper_context": dict(PAPER_CONTEXT, this_run_over_paper_gpu=value / PAPER_CONTEXT["gpu_moves_per_s"])}
        print(json.dumps({"bench_detail": detail}), flush=True)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": W["name"], "L": L, "samples": S, "runs_d_p": [list(r) for r in runs],
                           "mcs_per_step": mcs, "l2": "inputs > L2", "parallelism": f"group shards x{world}"},
                "roofline": compact_roofline(roofline),
                "cpu_baseline": None if cpu is None else dict(compact(cpu, ("value", "unit", "cores", "host_cores", "kind")),
                                                              sample=cpu["sample"].split(" (")[0]),
                "e2e": compact(e2e, ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")),
                "clocks": compact(clk, ("sm_mhz", "sm_max_mhz", "reasons")),
                "gpu_launches": launches,
                "batch": compact(batch, ("speedup", "batched", "plain", "results_identical", "frac")),
                "serving": None if serving is None else {
                    "capacity": serving["capacity"], "p50_latency_s": serving["p50_latency_s"],
                    "p99_latency_s": serving["p99_latency_s"], "at_load": serving["at_load"],
                    "curve": [[c["load"], round(c["throughput"] / 1e12, 3), round(c["p50_latency_s"], 4),
                               round(c["p99_latency_s"], 4)] for c in serving["curve"]]}}
        print(json.dumps(line, separators=(",", ":")), flush=True)
    for s in sims:
        s.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
