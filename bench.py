"""Benchmark of the sampled-space local-energy hot path on GB300.

One step = one pass of the whole path over one batch resident in HBM:
stage U (membership structure) -> FindCoupledPairs (count + fill, LoopOverTerms)
-> MatrixElement + ScatterAdd -> E_loc^var (FP32 compensated) -> E^var (FP64)
-> adjoint (pair-list VJP of L = E^var + sum_x g(x) E_loc^var(x)).
The Hamiltonian upload (grouping by XY) is set-up and not timed.

Workload (default): 56 qubits (28 orbitals, 14 electrons), ~2.3e5 Pauli terms,
1e5 peaked unique samples (the configuration the headline metric is quoted
on).  value = unique samples whose E_loc^var (and gradient) the step produced,
per second.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "unique-sample E_loc/s at 56 qubits (E_loc^var + E^var + adjoint per step)"
UNIT = "samples/s"
L2_FLUSH_BYTES = 512 << 20
SEARCH_SOURCE = os.path.join(ROOT, "paper_2408_07625_gb300", "csrc", "k_pairs.cu")
SEARCH_SECTION_END = "// CSR assembly:"  # the search kernel's source ends before this section
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "search_traffic.json")
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")
SM_COUNT, LANES_PER_SM, SM_MAX_GHZ = 152, 128, 2.07
OPS_PER_PROBE = 4  # algorithmic minimum per (sample, XY) probe: hash XOR, filter address, filter load, bit test


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload_config(inst, ham_info, n_pairs=None, schedule="terms", precision="fp32c"):
    cfg = {"workload": f"{inst.name}: {inst.n_qubits} qubits, {inst.n_alpha + inst.n_beta} electrons, "
                       f"{inst.n_terms} Pauli terms, {inst.n_unq} peaked unique samples",
           "n_qubits": inst.n_qubits, "n_terms": int(ham_info["n_terms"]), "n_xy": int(ham_info["n_xy"]),
           "n_unq": inst.n_unq, "schedule": schedule, "precision": precision,
           "l2": "flushed between timed steps (512 MiB write); inputs are smaller than L2"}
    if n_pairs is not None:
        cfg["n_pairs"] = int(n_pairs)
    return cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def search_source_sha256():
    """sha256 of the search kernel's source: k_pairs.cu up to its CSR-assembly
    section (staging, one-pass scratch and the LoopOverTerms search kernel)."""
    text = open(SEARCH_SOURCE, encoding="utf-8").read()
    return hashlib.sha256(text[:text.index(SEARCH_SECTION_END)].encode()).hexdigest()


def _profile_traffic():
    """Per-launch DRAM bytes of the search kernel from the committed ncu record
    (profiles/search_traffic.json), or None if absent or taken on a different
    kernel source."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    rec = json.load(open(PROFILE_TRAFFIC))
    if rec.get("search_source_sha256") != search_source_sha256():
        return None
    return float(rec["traffic_bytes_per_launch"])


def algorithmic_bytes(n, W, n_terms, n_xy, n_pairs, upstream=True):
    """HBM bytes one step must move by the path's data (no re-reads): U, log psi,
    E_loc (and the adjoint's upstream and gradient), the Hamiltonian tables
    (XY patterns with a 4-byte term offset, YZ mask and coefficient per term),
    and the pair list at 12 B per pair (i, j, pattern) written once by
    FindCoupledPairs and read once by E_loc^var and once by the adjoint."""
    per_sample = 8 * W + 8 + 8 + (16 if upstream else 0)
    return {"samples": n * per_sample, "hamiltonian": n_terms * (8 * W + 8) + n_xy * (8 * W + 4),
            "pairs": 12 * n_pairs * (3 if upstream else 2)}


def golden_rows(inst):
    """The oracle's per-row values for this workload (tests/golden/<name>_rows.npz,
    written by tests/golden/full_size.py), if stored for exactly this batch."""
    path = os.path.join(GOLDEN_DIR, f"{inst.name}_rows.npz")
    if not os.path.exists(path):
        return None
    g = np.load(path)
    sha = hashlib.sha256(np.ascontiguousarray(inst.U).tobytes()).hexdigest()
    if str(g["u_sha"]) != sha or len(g["eloc"]) != inst.n_unq:
        return None
    return g


def oriented_probes(U, xy, n_qubits):
    """(sample, pattern) probes of the oriented LoopOverTerms search: every
    non-diagonal pattern is probed by the samples on the rarer side (bit set
    or clear) of its highest qubit.  Host-side count from U and the patterns."""
    U = np.ascontiguousarray(U)
    n = U.shape[0]
    W = U.shape[1]
    occ = np.zeros(64 * W, np.int64)
    for w in range(W):
        bits = (U[:, w][:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
        occ[64 * w:64 * (w + 1)] = bits.sum(axis=0)
    side = np.where(2 * occ <= n, occ, n - occ)
    probes = 0
    for row in xy:
        top = -1
        for w in range(W - 1, -1, -1):
            if int(row[w]):
                top = 64 * w + int(row[w]).bit_length() - 1
                break
        if top >= 0:
            probes += int(side[top])
    return probes


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_baseline(inst, seconds=15.0, max_rows=None):
    """The oracle (pure Python, one core) on the first rows of the same batch."""
    import oracle
    t0 = time.time()
    ro = oracle.RowOracle.from_instance(inst)
    setup = time.time() - t0
    done = 0
    t0 = time.time()
    while time.time() - t0 < seconds and (max_rows is None or done < max_rows):
        ro.row(done)
        done += 1
    dt = time.time() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"E_loc^var of the first {done} rows of the same batch, LoopOverTerms per row in "
                      f"pure Python FP64 ({dt:.1f} s; oracle set-up {setup:.1f} s not timed)"}


def bench_full_eloc(nqs, torch, inst, n_sub, steps, warmup, flush, peak_gbs):
    """Exact local energy (Eq. local_energy) on the first n_sub samples of the
    batch: candidate generation with matrix elements and deduplication, then
    the sum over the candidates given their log-amplitudes (a seeded stand-in
    for the ansatz's values).  Device-timed with CUDA events on the stream."""
    dev = flush.device
    ham = nqs.Hamiltonian.from_instance(inst)
    U = torch.from_numpy(np.ascontiguousarray(inst.U[:n_sub]).view(np.int64)).to(dev)
    a = torch.from_numpy(inst.logpsi_re[:n_sub].copy()).to(dev)
    batch = nqs.Batch(ham, U, check=True)
    stream = torch.cuda.current_stream()
    fc = nqs.full_candidates(batch)
    ca = torch.from_numpy(np.random.default_rng(11).normal(-8.0, 2.0, fc.n_cand)).to(dev)
    er = torch.empty(n_sub, dtype=torch.float64, device=dev)
    for _ in range(warmup):
        fc = nqs.full_candidates(batch)
        nqs.local_energy_full(fc, a, None, ca, out=(er, None))
    torch.cuda.synchronize()
    t_gen, t_el = [], []
    for _ in range(steps):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        fc = nqs.full_candidates(batch)
        e1.record(stream)
        nqs.local_energy_full(fc, a, None, ca, out=(er, None))
        e2.record(stream)
        t_gen.append((e0, e1)); t_el.append((e1, e2))
    torch.cuda.synchronize()
    batch.status()
    ms_gen = float(np.mean([x.elapsed_time(y) for x, y in t_gen]))
    ms_el = float(np.mean([x.elapsed_time(y) for x, y in t_el]))
    n_xy = int(ham.info["n_xy"])
    entries = n_sub * n_xy
    W = inst.n_words
    # algorithmic bytes: per entry the candidate index (4 B) and matrix element (8 B) written by
    # the generation and read by the sum; per distinct candidate its key and U-index written and
    # its log-amplitude read; U, log psi and E_loc per sample; the Hamiltonian's XY table
    b_gen = entries * 12 + fc.n_cand * (8 * W + 4) + n_sub * (8 * W + 4) + n_xy * (8 * W + 4)
    b_el = entries * 12 + fc.n_cand * 8 + n_sub * 16
    roof = {"bound": "hbm", "kernel": "candidate generation (insert, compact, sort, relabel) + E_loc sum",
            "achieved": (b_gen + b_el) / ((ms_gen + ms_el) * 1e-3) / 1e9, "peak": peak_gbs, "unit": "GB/s",
            "frac": (b_gen + b_el) / ((ms_gen + ms_el) * 1e-3) / 1e9 / peak_gbs,
            "algorithmic_bytes": b_gen + b_el,
            "sum_only": {"achieved": b_el / (ms_el * 1e-3) / 1e9, "frac": b_el / (ms_el * 1e-3) / 1e9 / peak_gbs}}
    return {"workload": f"first {n_sub} samples of {inst.name}, {n_xy} XY patterns, {entries} candidate entries, "
                        f"{fc.n_cand} distinct candidates",
            "entries": entries, "n_cand": fc.n_cand, "ms_candidates": ms_gen, "ms_eloc_sum": ms_el,
            "entries_per_s": entries / ((ms_gen + ms_el) * 1e-3), "roofline": roof, "steps": steps}


def bench_sr(nqs, torch, n_sr, n_params, steps, flush, peaks):
    """min-SR step (Sec. "ANQS-tailored stochastic reconfiguration") on n_sr samples with
    n_params log-derivatives (synthetic FP32, seeded): top-probability selection is not
    included (the derivatives are the ansatz's, for the selected samples)."""
    dev = flush.device
    g = torch.Generator(device=dev).manual_seed(12)
    O = torch.randn((n_sr, n_params), generator=g, device=dev, dtype=torch.float32)
    O += torch.randn((1, n_params), generator=g, device=dev, dtype=torch.float32) * 0.5
    a = torch.randn(n_sr, generator=g, device=dev, dtype=torch.float64) * 0.7
    el = torch.randn(n_sr, generator=g, device=dev, dtype=torch.float64) - 5.0
    ev = torch.tensor([-5.1], dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        nqs.sr_step(O, a, el, ev, 1e-2)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nqs.sr_step(O, a, el, ev, 1e-2)
        e1.record(stream)
        ms.append((e0, e1))
    torch.cuda.synchronize()
    t = float(np.mean([x.elapsed_time(y) for x, y in ms]))
    o_bytes = 4.0 * n_sr * n_params
    # streamed form (n_params a multiple of 4): one M = 128, N = 256 MMA per K step ([hi hi^T | hi lo^T]);
    # otherwise three M = N = 128 MMAs (hi hi, hi lo, lo hi)
    mma_flops = (2.0 * 128 * 256 if n_params % 4 == 0 else 3 * 2.0 * 128 * 128) * n_params
    useful_flops = 2.0 * n_sr * n_sr * n_params
    return {"workload": f"N_SR = {n_sr} samples, {n_params} parameters (FP32 d log psi / d theta)",
            "ms_per_step": t,
            "hbm": {"bytes": 3 * o_bytes, "what": "O read by the mean, the Gram (tensor-core) and the step kernels",
                    "achieved_gbs": 3 * o_bytes / (t * 1e-3) / 1e9, "peak_gbs": peaks.get("hbm_gbs"),
                    "frac": 3 * o_bytes / (t * 1e-3) / 1e9 / peaks.get("hbm_gbs")},
            "tensor": {"mma_flops": mma_flops, "useful_flops": useful_flops,
                       "achieved_tflops": mma_flops / (t * 1e-3) / 1e12, "peak_tflops": peaks.get("bf16_tflops"),
                       "frac": mma_flops / (t * 1e-3) / 1e12 / peaks.get("bf16_tflops"),
                       "note": "over the whole step time (mean, Gram, FP64 sum and Cholesky solve, step)"}}


def bench_sampler(nqs, torch, n_qubits, K, steps, flush, peak_gbs):
    """Alg. 1 (ARGumbelTopK) over all n_qubits levels keeping K vectors: per
    level the extensions, their conditioned perturbed values, the ordering and
    the top-K cut (the library's kernels).  Two forms: the synchronous call per
    level (one host read of the kept count each), and the device-count form
    with the counts chained on the device, all levels captured once in a CUDA
    graph and replayed.  The ansatz's conditional log-probabilities are a
    seeded stand-in (log sigmoid of N(0, 2) logits, every outcome possible) and
    the Gumbel(0) draws are seeded; both are drawn before timing, one row per
    kept vector."""
    dev = flush.device
    W = (n_qubits + 63) // 64
    g = torch.Generator(device=dev).manual_seed(13)
    z = torch.randn((n_qubits, K), generator=g, device=dev, dtype=torch.float64) * 2.0
    logp = torch.stack([torch.nn.functional.logsigmoid(z), torch.nn.functional.logsigmoid(-z)], dim=2).contiguous()
    u = torch.rand((n_qubits, K, 2), generator=g, device=dev, dtype=torch.float64).clamp_min(1e-300)
    G = (-torch.log(-torch.log(u))).contiguous()
    del z, u
    bufs = [(torch.empty((K, W), dtype=torch.int64, device=dev), torch.empty(K, dtype=torch.float64, device=dev),
             torch.empty(K, dtype=torch.float64, device=dev)) for _ in range(2)]
    lib = nqs.load_library()
    scratch = torch.empty(int(lib.nqs_gumbel_scratch_bytes(K)), dtype=torch.uint8, device=dev)
    zero = torch.zeros(1, dtype=torch.float64, device=dev)
    one = torch.ones(1, dtype=torch.int64, device=dev)
    counts = torch.zeros((n_qubits, 2), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    sizes = []

    def run_sync():
        x, l, lt = None, zero, zero
        sizes.clear()
        for i in range(n_qubits):
            n = int(l.shape[0])
            x, l, lt = nqs.gumbel_topk_level(n_qubits, i, x, l, lt, logp[i, :n], G[i, :n], K, out=bufs[i & 1],
                                             scratch=scratch)
            sizes.append(n)
        return int(l.shape[0])

    def run_async():
        x, l, lt, n_dev, max_n = None, zero, zero, one, 1
        for i in range(n_qubits):
            out = bufs[i & 1]
            nqs.gumbel_topk_level_async(n_qubits, i, max_n, n_dev, x, l, lt, logp[i], G[i], K, out, scratch, counts[i])
            x, l, lt, n_dev = out[0], out[1], out[2], counts[i]
            max_n = min(K, 2 * max_n)

    def timed(fn):
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            ms.append((e0, e1))
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ms]))

    for _ in range(3):
        run_sync()
    torch.cuda.synchronize()
    t_sync = timed(run_sync)
    kept = min(K, 2 * sizes[-1])
    # the device-count form, captured once (after a warm-up on the capture's side stream)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        run_async()
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        run_async()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    t_graph = timed(graph.replay)
    status = counts[:, 1].cpu().numpy()
    kept_graph = int(counts[-1, 0].item())
    # algorithmic bytes per level: each parent's words, l, L~, two log-probabilities and two
    # draws read; each kept child's words, l' and L~' written
    outs = sizes[1:] + [kept]
    bytes_ = sum(n * (8 * W + 16 + 32) + o * (8 * W + 16) for n, o in zip(sizes, outs))
    return {"workload": f"{n_qubits} qubits, K = {K} kept vectors, {sum(sizes)} parents over {n_qubits} levels",
            "ms_per_sampling": t_graph, "us_per_level": 1e3 * t_graph / n_qubits,
            "samples_per_s": kept_graph / (t_graph * 1e-3),
            "form": "device-held counts, all levels in one CUDA graph (4 kernels a level, no host round trip)",
            "levels_ok": int((status == 1).sum()), "kept": kept_graph,
            "sync_form": {"ms_per_sampling": t_sync, "samples_per_s": kept / (t_sync * 1e-3),
                          "what": "one library call per level through the Python binding, each reading the kept "
                                  "count back to the host"},
            "hbm": {"bytes": bytes_, "achieved_gbs": bytes_ / (t_graph * 1e-3) / 1e9, "peak_gbs": peak_gbs,
                    "frac": bytes_ / (t_graph * 1e-3) / 1e9 / peak_gbs,
                    "note": "the working set stays in L2; the levels are latency-bound (see the profile summary)"},
            "steps": steps}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    from synth import config_instance
    inst = config_instance(args.workload, n_unq=args.n_unq)
    import oracle
    ro = oracle.RowOracle.from_instance(inst)
    rows_per_step = args.ref_rows
    nxt = 0
    for _ in range(args.warmup):
        for _ in range(rows_per_step):
            ro.row(nxt % inst.n_unq); nxt += 1
    t0 = time.time()
    for _ in range(args.steps):
        for _ in range(rows_per_step):
            ro.row(nxt % inst.n_unq); nxt += 1
    dt = time.time() - t0
    value = args.steps * rows_per_step / dt
    xm = np.ascontiguousarray(inst.x_mask).reshape(len(inst.x_mask), -1)
    n_xy = len(np.unique(xm, axis=0))
    # the same workload description as the GPU arm's line; the oracle runs in FP64 on the host
    ref_config = _workload_config(inst, {"n_terms": inst.n_terms, "n_xy": n_xy}, schedule="terms",
                                  precision="fp64")
    ref_config["l2"] = "host run: no GPU caches involved"
    ref_config["sample_rows_per_step"] = rows_per_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": ref_config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{rows_per_step} rows of the batch per step (pure Python FP64 oracle, "
                                       "LoopOverTerms per row)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2408_07625_gb300 as nqs
    from synth import config_instance

    inst = config_instance(args.workload, n_unq=args.n_unq)
    ham = nqs.Hamiltonian.from_instance(inst)
    n = inst.n_unq
    U_host = torch.from_numpy(np.ascontiguousarray(inst.U).view(np.int64)).pin_memory()
    a_host = torch.from_numpy(inst.logpsi_re.copy()).pin_memory()
    U = U_host.to(dev)
    a = a_host.to(dev)
    rng = np.random.default_rng(7)
    g_host = torch.from_numpy(rng.normal(0, 1e-3, size=n)).pin_memory()
    g = g_host.to(dev)
    gE = torch.ones(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    prec = args.precision
    batch = nqs.Batch(ham, U, check=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    ev = {k: [] for k in ("stage", "pairs", "energy", "evar", "backward")}
    # rows of this rank: one contiguous block balanced by pair counts (all rows on one GPU)
    r0, r1 = 0, n
    bounds = [0, n]
    if ws > 1:
        from paper_2408_07625_gb300.sharding import row_blocks, combine_evar, sharded_coupled_pairs
        rp_all, _ = nqs.count_pairs(batch)
        blocks = row_blocks(rp_all.cpu().numpy(), ws)
        bounds = [b[0] for b in blocks] + [n]
        r0, r1 = blocks[rank]

    hbuf = [None]  # per-pair matrix elements, kept from E_loc^var for the adjoint
    cap = [None]   # pair capacity for the no-wait search (set by the first step)
    # outputs allocated once (every row of the range is written by each call)
    outs = {"e": (torch.zeros(n, dtype=torch.float64, device=dev), None,
                  torch.zeros(n, dtype=torch.float64, device=dev)),
            "g": (torch.zeros(n, dtype=torch.float64, device=dev), None),
            "v": torch.zeros(3, dtype=torch.float64, device=dev)}

    def step(batch_obj, Udev, adev, record=False, prec=prec):
        marks = []
        def mark():
            if record:
                e = torch.cuda.Event(enable_timing=True); e.record(stream); marks.append(e)
        mark()
        batch_obj.restage(Udev)
        mark()
        if ws > 1 and args.schedule == "terms":
            # sharded search: this rank's slice of the work items, records exchanged to the row owners
            rp, pj, pk = sharded_coupled_pairs(batch_obj, bounds, rank, ws)
        elif cap[0] is None:
            # rows as the search placed them: the energy and adjoint sums are exact, so no row sort
            rp, pj, pk = nqs.coupled_pairs(batch_obj, r0, r1, schedule=args.schedule, reuse=True, sort_rows=False)
            cap[0] = int(pj.numel() * 1.02) + 1024   # the list size of this batch, for the no-wait form
        else:
            # no host wait: the buffers are sized from the first call; an overflow would show in
            # the workspace status, which is checked after the timed steps
            rp, pj, pk = nqs.coupled_pairs_async(batch_obj, cap[0], r0, r1, schedule=args.schedule,
                                                 sort_rows=False, packed=args.schedule == "terms")
        total = int(pj.numel())
        mark()
        hdt = torch.float64 if prec == "fp64" else torch.float32
        if hbuf[0] is None or hbuf[0].dtype != hdt or hbuf[0].numel() < (2 if prec == "fp32c" else 1) * total:
            hbuf[0] = nqs.pair_h_buffer(int(total * 1.1) + 1024, prec, dev)
        hp = hbuf[0][:total] if total > 0 else None
        er, ei, hd = nqs.local_energy(batch_obj, adev, None, (rp, pj, pk), prec, r0, r1, out=outs["e"],
                                      hpair=hp)
        mark()
        evar = nqs.variational_energy(batch_obj, adev[r0:r1], er[r0:r1], out=outs["v"])
        if ws > 1:  # the one exchange: every rank's [E, max, sum] triple
            evar = combine_evar(evar)
        mark()
        gr, gi = nqs.local_energy_backward(batch_obj, adev, None, er, ei, hd, evar, g, None, gE,
                                           (rp, pj, pk), prec, r0, r1, out=outs["g"], hpair=hp)
        mark()
        return er, evar, gr, total, marks

    for _ in range(args.warmup):
        step(batch, U, a)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    nqs.search_time()  # drop any earlier intervals
    nqs.search_timing(args.schedule == "terms")
    starts, ends = [], []
    total_pairs = 0
    for it in range(args.steps):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True); s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        er, evar, gr, total_pairs, marks = step(batch, U, a, record=True)
        s1.record(stream)
        starts.append(s0); ends.append(s1)
        for name, (m0, m1) in zip(ev.keys(), zip(marks[:-1], marks[1:])):
            ev[name].append((m0, m1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    nqs.search_timing(False)
    search_ms, search_launches = nqs.search_time()
    batch.status()  # the no-wait searches of the timed steps all fit their buffers
    if ws == 1 or args.schedule != "terms":
        # the pair count of the batch (the buffers of the no-wait search are larger)
        total_pairs = int(batch._async_rp[-1]) if batch._async_rp is not None else total_pairs
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_ms = float(np.sum(step_ms))
    if ws > 1:
        t = torch.tensor([t_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_ms = float(t.item())
        torch.distributed.barrier()
    ms_per_step = t_ms / args.steps
    value = ws * n * args.steps / (t_ms * 1e-3)
    phases = {k: float(np.mean([m0.elapsed_time(m1) for m0, m1 in v])) for k, v in ev.items()}

    # the same step captured once in a CUDA graph and replayed: the library calls of a step
    # enqueue no host work and no host wait, so one replay runs the whole step (no launch gaps);
    # this is the headline figure, the eager loop above gives the phases and the search timing
    graph = None
    if ws == 1:
        try:
            side = torch.cuda.Stream()
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                step(batch, U, a)
            stream.wait_stream(side)
            torch.cuda.synchronize()
            g_step = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g_step):
                step(batch, U, a)
            for _ in range(max(3, args.warmup)):
                g_step.replay()
            torch.cuda.synchronize()
            g_clocks = ClockSampler(local)
            g_clocks.start()
            time.sleep(0.3)
            g_ev = []
            for it in range(args.steps):
                flush.zero_()
                s0 = torch.cuda.Event(enable_timing=True); s1 = torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                g_step.replay()
                s1.record(stream)
                g_ev.append((s0, s1))
            torch.cuda.synchronize()
            g_clk = g_clocks.stop()
            batch.status()  # every replayed search fitted its buffers
            g_ms = float(np.sum([s0.elapsed_time(s1) for s0, s1 in g_ev]))
            graph = {"ms_per_step": g_ms / args.steps, "clocks": g_clk}
            del g_step
        except Exception as exc:  # reported in the line; the eager figure stays the headline
            graph = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    eager_ms_per_step = ms_per_step
    if graph is not None and "ms_per_step" in graph:
        ms_per_step = graph["ms_per_step"]
        value = n / (ms_per_step * 1e-3)
        clk = graph["clocks"]

    # the half-stored pair path (each unordered pair once, symmetric scatter), same batch and rules
    def step_half(batch_obj, Udev, adev):
        batch_obj.restage(Udev)
        half = nqs.half_pairs(batch_obj)
        if hbuf_half[0] is None or hbuf_half[0].shape[0] < half[3]:
            hbuf_half[0] = nqs.half_h_buffer(int(half[3] * 1.1) + 1024, prec, dev)
        hr = hbuf_half[0][:half[3]]
        er, ei, hd = nqs.local_energy_half(batch_obj, adev, None, half, prec, out=outs["e"], hrec=hr)
        evar = nqs.variational_energy(batch_obj, adev, er, out=outs["v"])
        gr, gi = nqs.local_energy_backward_half(batch_obj, adev, None, er, ei, hd, evar, g, None, gE, half, prec,
                                                hrec=hr, out=outs["g"])
        return er, evar, gr

    half_ms = None
    if ws == 1:
        hbuf_half = [None]
        for _ in range(3):
            step_half(batch, U, a)
        torch.cuda.synchronize()
        h_ev = []
        for it in range(args.steps):
            flush.zero_()
            s0 = torch.cuda.Event(enable_timing=True); s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            er_h, ev_h, gr_h = step_half(batch, U, a)
            s1.record(stream)
            h_ev.append((s0, s1))
        torch.cuda.synchronize()
        half_ms = float(np.mean([s0.elapsed_time(s1) for s0, s1 in h_ev]))

    # the other precision on the same batch, same step, same timing rules
    other = "fp64" if prec == "fp32c" else "fp32c"
    for _ in range(3):
        step(batch, U, a, prec=other)
    torch.cuda.synchronize()
    o_ms = []
    for it in range(args.steps):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True); s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        step(batch, U, a, prec=other)
        s1.record(stream)
        o_ms.append((s0, s1))
    torch.cuda.synchronize()
    other_ms = float(np.mean([s0.elapsed_time(s1) for s0, s1 in o_ms]))
    if ws > 1:
        t = torch.tensor([other_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        other_ms = float(t.item())

    # e2e: public API with host buffers (H2D of U and log psi, D2H of E_loc, gradient, E^var)
    out_e = torch.empty(n, dtype=torch.float64).pin_memory()
    out_g = torch.empty(n, dtype=torch.float64).pin_memory()
    out_v = torch.empty(3, dtype=torch.float64).pin_memory()
    U2 = torch.empty_like(U); a2 = torch.empty_like(a)
    batch2 = nqs.Batch(ham, U, check=True)
    U2.copy_(U); a2.copy_(a)
    e_graph = None
    if graph is not None and "ms_per_step" in graph:
        # as the headline: the step on the copied-in buffers captured once, replayed each step
        er, evar, gr, _, _ = step(batch2, U2, a2)   # sizes the no-wait search's buffers
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            step(batch2, U2, a2)
        stream.wait_stream(side)
        torch.cuda.synchronize()
        e_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(e_graph):
            er, evar, gr, _, _ = step(batch2, U2, a2)
        for _ in range(3):
            e_graph.replay()
        torch.cuda.synchronize()
    e_starts, e_ends = [], []
    for it in range(args.steps):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True); s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        U2.copy_(U_host, non_blocking=True)
        a2.copy_(a_host, non_blocking=True)
        if e_graph is not None:
            e_graph.replay()
        else:
            er, evar, gr, _, _ = step(batch2, U2, a2)
        out_e[r0:r1].copy_(er[r0:r1], non_blocking=True)
        out_g[r0:r1].copy_(gr[r0:r1], non_blocking=True)
        out_v.copy_(evar, non_blocking=True)
        s1.record(stream)
        e_starts.append(s0); e_ends.append(s1)
    torch.cuda.synchronize()
    batch2.status()
    e2e_ms = float(np.sum([s.elapsed_time(e) for s, e in zip(e_starts, e_ends)]))
    if ws > 1:
        t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = ws * n * args.steps / (e2e_ms * 1e-3)
    h2d = U.numel() * 8 + a.numel() * 8
    d2h = (r1 - r0) * 8 * 2 + 3 * 8

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # FP32C vs FP64 (untimed), and both against the oracle's values of every row when stored
    r64 = nqs.evaluate(batch, a, None, "fp64", schedule=args.schedule)
    r32 = nqs.evaluate(batch, a, None, "fp32c", schedule=args.schedule)
    err = {"fp32c_vs_fp64_gpu": {"max_abs_dE_loc": float((r64["eloc_re"] - r32["eloc_re"]).abs().max().item()),
                                 "abs_dE_var": abs(float(r64["evar"][0].item()) - float(r32["evar"][0].item()))},
           "E_var_fp64": float(r64["evar"][0].item())}
    gold = golden_rows(inst) if (r0, r1) == (0, n) else None
    if gold is not None:
        for name, r in (("fp64", r64), ("fp32c", r32)):
            d = np.abs(r["eloc_re"].cpu().numpy() - gold["eloc"])
            err[f"{name}_vs_oracle"] = {"max_abs_dE_loc": float(d.max()), "mean_abs_dE_loc": float(d.mean()),
                                        "abs_dE_var": abs(float(r["evar"][0].item()) - float(gold["evar"][0])),
                                        "rows": int(len(d))}
        err["oracle"] = ("FP64 CPU oracle, every row (tests/golden/" + inst.name + "_rows.npz, written by "
                         "tests/golden/full_size.py)")
        err["oracle_E_var"] = float(gold["evar"][0])

    # roofline of the dominant kernel: the LoopOverTerms search (one launch per step),
    # against the integer peak measured on this GPU by the library's microbenchmark
    info = ham.info
    derived = SM_COUNT * LANES_PER_SM * SM_MAX_GHZ * 1e9 / 1e12
    alu_peak, loop_peak = nqs.probe_peaks()
    if search_launches > 0:
        xy = ham.export()[0]
        probes = oriented_probes(inst.U, xy, inst.n_qubits)
        launch_ms = search_ms / search_launches
        achieved = OPS_PER_PROBE * probes / (launch_ms * 1e-3) / 1e12
        peak = alu_peak / 1e12
        roof = {"bound": "alu", "kernel": "pairs_terms_kernel (oriented LoopOverTerms search)",
                "achieved": achieved, "peak": peak,
                "unit": "Tops/s (integer lane-ops; 4 per sample-pattern probe)", "frac": achieved / peak,
                "traffic": _profile_traffic(), "launch_ms": launch_ms, "probes_per_launch": probes,
                "launches_timed": search_launches,
                "peak_source": "measured: nqs_probe_peaks register-only XOR/AND/funnel-shift mix, "
                               "152 x 1024 threads, CUDA events (derived unit-count figure: "
                               f"{derived:.1f} Tops/s)",
                "probe_loop": {"achieved_gprobes_s": probes / (launch_ms * 1e-3) / 1e9,
                               "peak_gprobes_s": loop_peak / 1e9,
                               "frac": probes / (launch_ms * 1e-3) / loop_peak,
                               "peak_source": "measured: the search's filter loop alone (128 KB shared "
                                              "filter, no survivors), nqs_probe_peaks"}}
    else:
        roof = None
    peaks, src = _peaks()
    ab = algorithmic_bytes(r1 - r0, inst.n_words, int(info["n_terms"]), int(info["n_xy"]), total_pairs)
    ab_total = float(sum(ab.values()))
    hbm = {"algorithmic_bytes_per_step": ab_total, "parts": ab,
           "achieved_gbs": ab_total / (ms_per_step * 1e-3) / 1e9, "peak_gbs": peaks.get("hbm_gbs"),
           "frac": ab_total / (ms_per_step * 1e-3) / 1e9 / peaks.get("hbm_gbs"),
           "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback",
           "model": "U, log psi, E_loc, upstream, gradient: (8W + 32) B per sample; Hamiltonian: (8W + 8) B "
                    "per term + (8W + 4) B per XY pattern; pair list 12 B per pair written once and read "
                    "twice (E_loc^var, adjoint)"}
    # library kernels per step: staging (hash table and filter, per-qubit lists), the pairs phase
    # (terms: count init, search, 3-kernel scan, row init, scatter into packed pair words (no row sort);
    # batch: count, scan, fill; trie: tree build, count, scan, fill), then amplitudes + row order (2)
    # + E_loc^var, E^var (+ combination across ranks), amplitudes + adjoint weights + row order (2)
    # + adjoint
    pairs_kernels = {"terms": 2 + 1 + 1 + 3 + 1 + 1 + 1, "batch": 2 + 1 + 3 + 1,
                     "trie": 2 + 3 * ((inst.n_qubits + 7) // 8) + 7 + 1 + 3 + 1}[args.schedule]
    if ws > 1 and args.schedule == "terms":
        # sharded: staging, search slice, routing (count, scatter), record counts (init, count),
        # 3-kernel scan, row init, scatter, warp and block row sorts
        pairs_kernels = 2 + 1 + 2 + 2 + 3 + 1 + 1 + 2
    kernels_per_step = pairs_kernels + 4 + 1 + (1 if ws > 1 else 0) + 5
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "u64+f32c (FP32 compensated, FP64 reduction)" if prec == "fp32c" else "u64+f64",
            "data": "synthetic (seeded integrals, JW, peaked samples)",
            "config": dict(_workload_config(inst, info, total_pairs, args.schedule, prec),
                           parallelism=f"search work items sharded over {ws} GPU(s), records all-to-all to the row owners; rows sharded; E^var triples all-gathered" if ws > 1
                           else "one GPU", rows_rank0=[r0, r1]),
            "timing": ("one CUDA graph replay per step (the step captured once; L2 flushed before each replay)"
                       if eager_ms_per_step != ms_per_step else "library calls launched step by step"),
            "eager_ms_per_step": eager_ms_per_step,
            "graph_error": graph.get("error") if graph else None,
            "pairs_per_s": total_pairs / (phases["pairs"] * 1e-3),
            "phases_ms": phases, "precision_error": err,
            f"{other}_ms_per_step": other_ms,
            f"{other}_value": ws * n / (other_ms * 1e-3),
            "half_pairs_path": None if half_ms is None else {
                "ms_per_step": half_ms, "value": n / (half_ms * 1e-3), "unit": UNIT,
                "what": "same step with each unordered pair stored once (i, j, k) and both rows updated by FP64 "
                        "atomic addition (no scatter, no row sort; one matrix element per unordered pair)",
                "precision": prec},
            "roofline": roof, "hbm": hbm,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": kernels_per_step * args.steps,
            "clocks": clk}
    if ws == 1 and args.sr_params > 0:
        line["sr"] = bench_sr(nqs, torch, 100, args.sr_params, max(3, args.steps // 4), flush, peaks)
    if ws == 1 and not args.no_batch64:
        b = measure_batched(args, steps=max(3, args.steps // 3), gradients=True)
        line["batch64"] = {k: b[k] for k in ("metric", "value", "unit", "ms_per_step", "config", "sequential_ms_per_step",
                                             "e2e", "gpu_launches", "tuned", "gradients")}
    if ws == 1 and args.full_n > 0:
        line["full_eloc"] = bench_full_eloc(nqs, torch, inst, min(args.full_n, n), max(3, args.steps // 4), 3, flush,
                                            peaks.get("hbm_gbs"))
    if ws == 1 and args.sampler_k > 0:
        line["sampler"] = bench_sampler(nqs, torch, inst.n_qubits, args.sampler_k, max(3, args.steps // 4), flush,
                                        peaks.get("hbm_gbs"))
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(inst, seconds=args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


BATCH_METRIC = ("unique-sample E_loc/s over 64 batched instances of 20-56 qubits (E_loc^var + E^var, and with "
                "gradients dE^var/dlog psi, one graph)")


def run_sr_only(args):
    """The min-SR step alone (``--sr-only``): one JSON line with the SR measurement."""
    import torch
    torch.cuda.set_device(0)
    import paper_2408_07625_gb300 as nqs
    peaks, _ = _peaks()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    sr = bench_sr(nqs, torch, 100, args.sr_params, args.steps, flush, peaks)
    print(json.dumps(dict(sr, metric="min-SR step time (N_SR = 100)", unit="ms", higher_is_better=False,
                          value=sr["ms_per_step"], steps=args.steps)), flush=True)


def run_sampler_only(args):
    """ARGumbelTopK alone (``--sampler-only``): one JSON line with the sampler measurement."""
    import torch
    torch.cuda.set_device(0)
    import paper_2408_07625_gb300 as nqs
    peaks, _ = _peaks()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    sm = bench_sampler(nqs, torch, args.sampler_qubits, args.sampler_k, args.steps, flush, peaks.get("hbm_gbs"))
    print(json.dumps(dict(sm, metric="ARGumbelTopK samples/s", unit="samples/s", higher_is_better=True,
                          value=sm["samples_per_s"], steps=args.steps)), flush=True)


def run_batched(args):
    """All instances of the batched workload evaluated by one CUDA-graph launch per step."""
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    line = measure_batched(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def measure_batched(args, ws=1, rank=0, local=0, steps=None, gradients=False):
    """The batched workload's measurements (a dict; rank 0's values)."""
    import torch
    dev = torch.device("cuda", local)
    import paper_2408_07625_gb300 as nqs
    from synth import batched_instances
    steps = args.steps if steps is None else steps

    insts = batched_instances(64)
    hams = {}
    items, hosts = [], []
    for inst in insts:
        if inst.n_qubits not in hams:
            hams[inst.n_qubits] = nqs.Hamiltonian.from_instance(inst)
        Uh = torch.from_numpy(np.ascontiguousarray(inst.U).view(np.int64)).pin_memory()
        ah = torch.from_numpy(inst.logpsi_re.copy()).pin_memory()
        hosts.append((Uh, ah))
        items.append((hams[inst.n_qubits], Uh.to(dev), ah.to(dev)))
    t0 = time.time()
    plan = nqs.BatchedPlan(items, precision=args.precision, autotune=True, gradients=gradients)
    t_plan = time.time() - t0
    total = sum(inst.n_unq for inst in insts)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        plan.run()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record(stream); plan.run(); b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_ms = float(sum(a.elapsed_time(b) for a, b in ev))
    rc, bad = plan.status()
    if rc != 0:
        raise SystemExit(f"instance {bad} failed with status {rc}")
    # the same kernels launched instance by instance (no graph), for comparison
    batches = [nqs.Batch(it[0], it[1]) for it in items]
    scheds = [plan.info(i)["schedule"] for i in range(len(items))]
    seq = []
    for _ in range(max(1, steps // 3)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for bt, it, sch in zip(batches, items, scheds):
            bt.restage()
            nqs.evaluate(bt, it[2], None, args.precision, schedule=sch, keep_pairs=False)
        b.record(stream)
        seq.append((a, b))
    torch.cuda.synchronize()
    seq_ms = float(np.mean([a.elapsed_time(b) for a, b in seq]))
    # end to end: pinned host inputs in, E_loc and E^var out, every step
    outs = [(torch.empty(inst.n_unq, dtype=torch.float64).pin_memory(), torch.empty(3, dtype=torch.float64).pin_memory(),
             torch.empty(inst.n_unq, dtype=torch.float64).pin_memory() if gradients else None) for inst in insts]
    e2e = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i, (Uh, ah) in enumerate(hosts):
            plan.U[i].copy_(Uh, non_blocking=True)
            plan.logpsi[i].copy_(ah, non_blocking=True)
        plan.run()
        for i, (oe, ov, og) in enumerate(outs):
            oe.copy_(plan.eloc[i], non_blocking=True)
            ov.copy_(plan.evar[i], non_blocking=True)
            if og is not None:
                og.copy_(plan.grad[i], non_blocking=True)
        b.record(stream)
        e2e.append((a, b))
    torch.cuda.synchronize()
    e2e_ms = float(sum(a.elapsed_time(b) for a, b in e2e))
    if ws > 1:
        t = torch.tensor([t_ms, e2e_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_ms, e2e_ms = float(t[0].item()), float(t[1].item())
    h2d = sum(inst.U.nbytes + inst.logpsi_re.nbytes for inst in insts)
    d2h = sum(8 * inst.n_unq * (2 if gradients else 1) + 24 for inst in insts)
    counts = {k: scheds.count(k) for k in sorted(set(scheds))}
    n_pairs = int(sum(plan.info(i)["planned_pairs"] for i in range(len(items))))
    line = {"metric": BATCH_METRIC, "value": ws * total * steps / (t_ms * 1e-3), "unit": UNIT,
            "n_gpus": ws, "steps": steps, "warmup": args.warmup, "ms_per_step": t_ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64+f32c (FP32 compensated, FP64 reduction)" if args.precision == "fp32c" else "u64+f64",
            "data": "synthetic (seeded integrals, JW, peaked samples)",
            "config": {"workload": f"batched: 64 instances, N in {{20,28,36,44,56}}, {total} samples in all, "
                                   f"{n_pairs} pairs", "instances": len(items), "n_unq_total": total,
                       "n_pairs": n_pairs, "schedules": counts, "graph_nodes": plan.info(0)["graph_nodes"],
                       "plan_s": round(t_plan, 2), "precision": args.precision,
                       "l2": "flushed between timed steps (512 MiB write)"},
            "sequential_ms_per_step": seq_ms,
            "e2e": {"value": ws * total * steps / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": plan.info(0)["graph_kernels"] * steps, "clocks": clk,
            "tuned": {"schedules": counts,
                      "terms_settings": sorted({(plan.info(i)["tune"]["terms_grab"], plan.info(i)["tune"]["terms_groups"])
                                                for i in range(len(items)) if scheds[i] == "terms"}),
                      "trie_settings": sorted({plan.info(i)["tune"]["trie_pop"] for i in range(len(items))
                                               if scheds[i] == "trie"})},
            "gradients": gradients}
    return line


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="h56")
    p.add_argument("--n-unq", type=int, default=None, help="smaller peaked batch of the same Hamiltonian")
    p.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"])
    p.add_argument("--schedule", default="terms", choices=["terms", "batch", "trie"])
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--ref-rows", type=int, default=40)
    p.add_argument("--sr-params", type=int, default=1_000_000,
                   help="parameters of the min-SR measurement (100 samples); 0 skips it")
    p.add_argument("--no-batch64", action="store_true", help="skip the 64-instance batched measurement")
    p.add_argument("--sr-only", action="store_true", help="time only the min-SR step (--sr-params parameters)")
    p.add_argument("--sampler-k", type=int, default=100_000,
                   help="vectors kept per level by the ARGumbelTopK measurement; 0 skips it")
    p.add_argument("--sampler-only", action="store_true",
                   help="time only the ARGumbelTopK sampler (--sampler-qubits levels, --sampler-k kept)")
    p.add_argument("--sampler-qubits", type=int, default=56)
    p.add_argument("--full-n", type=int, default=1000,
                   help="samples of the exact-local-energy (Eq. local_energy) measurement; 0 skips it")
    args = p.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.sr_only:
        run_sr_only(args)
    elif args.sampler_only:
        run_sampler_only(args)
    elif args.workload == "batch64":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
