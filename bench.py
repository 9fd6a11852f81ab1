"""Benchmark of the convolution-product expansion apply (Eq. 1.4) and its adjoint.

One step = one forward apply y = H_m u and one adjoint apply x = H_m^* u of a
whole batch of right-hand sides (every kernel of the hot path runs once per
chunk of the batch).  Metric: applies per second, counting each right-hand
side of each direction as one apply.

Default workload: 2D periodic 1024 x 1024 float32 images, batch 8, m = 16
bilinear hat windows on a 4 x 4 node grid, anisotropic rotated Gaussian PSFs
(sigma_x = 1.5 + y1, sigma_y = 1.5 + y2 px, theta = pi y1 y2), u ~ U[0,1).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Under torchrun (N > 1) every rank runs its own batch (weak scaling: the
right-hand sides are independent, no data-path collective), the step time is
the max over ranks and rank 0 prints the JSON line.  ``--impl reference``
times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "H·u and H*·v applies/sec (fused FP32 path, rel-l2 <= 1e-5 vs FP64 oracle)"
UNIT = "applies/s"
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128


# DRAM bytes (read + write) per launch measured by ncu for the dominant kernels
# of the 1024 x 1024, m = 16, B = 8 workload with tensor-product windows (one
# launch = 8 right-hand sides); see profiles/kw_cols_2d_1024_m16_b8.md.  Valid
# only for that workload and the kernels as captured.
MEASURED_TRAFFIC = {("2d_1024x1024_m16_b8", "separable", "cols_fwd"): 207.906304e6 + 18.656512e6,
                    ("2d_1024x1024_m16_b8", "separable", "cols_adj"): 102.050816e6 + 89.044224e6}

# ------------------------------------------------------------- algorithmic work

def cyclic_extent(flags) -> tuple[int, int]:
    """(start, length) of the shortest periodic interval holding every set flag."""
    n = len(flags)
    if not np.any(flags):
        return 0, 0
    if np.all(flags):
        return 0, n
    best = run = 0
    best_end = 0
    for t in range(2 * n):
        if not flags[t % n]:
            run += 1
            if run > best and run <= n:
                best, best_end = run, t
        else:
            run = 0
    return (best_end + 1) % n, n - best


def slot_boxes(wy: np.ndarray, wx: np.ndarray) -> list:
    """Boxes (r0, nr, c0, nc) of the row-transform slots of a separable plan: one
    per distinct column factor, rows = union of its terms' row supports."""
    slots = {}
    for k in range(wy.shape[0]):
        slots.setdefault(wx[k].tobytes(), []).append(k)
    out = []
    for key, ks in slots.items():
        rows = np.any(wy[ks] != 0, axis=0)
        r0, nr = cyclic_extent(rows)
        c0, nc = cyclic_extent(wx[ks[0]] != 0)
        out.append((r0, nr, c0, nc))
    return out


def work_model(pr: synth.Problem, boxes, nb: int, slots=None) -> dict:
    """Algorithmic flops and bytes per launch of each kernel kind for a chunk of nb right-hand sides.

    Flops are the nominal FFT counts (5 N log2 N per complex N-point FFT,
    2.5 N log2 N per real one), 8 per complex multiply-add, 1 per window
    multiply.  Bytes are the compulsory global traffic of the kernel: its
    inputs read once and its outputs written once.  With `slots` (separable
    windows) the row passes transform one row set per slot instead of one per
    term, the column passes multiply by the row factors.
    """
    if len(pr.shape) == 1:
        n = pr.shape[0]
        m = pr.m
        fft_r = 2.5 * n * math.log2(n)
        fl = nb * (m * (fft_r + n + 8 * (n // 2 + 1)) + fft_r)
        by = nb * n * 8 + m * (n // 2 + 1) * 8 + m * n * 4
        return {"fwd_1d": (fl, by), "adj_1d": (fl, by)}
    ny, nx = pr.shape
    m = pr.m
    nxh = nx // 2
    rows = sum(b[1] for b in boxes)
    box_px = sum(b[1] * b[3] for b in boxes)
    lx, ly = math.log2(nx), math.log2(ny)
    f_row_r2c = 2.5 * nx * lx
    f_col = 5.0 * ny * ly
    hbytes = m * ny * (nxh + 1) * 8
    zbytes = nb * rows * nxh * 8
    abytes = nb * ny * nxh * 8
    ubytes = nb * ny * nx * 4
    if slots:
        srows = sum(b[1] for b in slots)
        spx = sum(b[1] * b[3] for b in slots)
        sbytes = nb * srows * nxh * 8
        wcols = sum(b[3] for b in slots) * 4
        cfl = nb * ((m + 1) * (nxh + 1) * f_col + m * 8 * ny * (nxh + 1) + rows * (nxh + 1) * 2)
        return {
            "rows_r2c_window": (nb * (srows * f_row_r2c + spx), ubytes + wcols + sbytes),
            "cols_fwd": (cfl, sbytes + hbytes + abytes + m * ny * 4),
            "rows_c2r": (nb * ny * f_row_r2c, abytes + ubytes),
            "rows_r2c": (nb * ny * f_row_r2c, ubytes + abytes),
            "cols_adj": (cfl, abytes + hbytes + sbytes + m * ny * 4),
            "rows_adj": (nb * (srows * f_row_r2c + spx), sbytes + wcols + ubytes),
        }
    return {
        "rows_r2c_window": (nb * (rows * f_row_r2c + box_px), ubytes + box_px * 4 + zbytes),
        "cols_fwd": (nb * ((m + 1) * (nxh + 1) * f_col + m * 8 * ny * (nxh + 1)),
                     zbytes + hbytes + abytes),
        "rows_c2r": (nb * ny * f_row_r2c, abytes + ubytes),
        "rows_r2c": (nb * ny * f_row_r2c, ubytes + abytes),
        "cols_adj": (nb * ((m + 1) * (nxh + 1) * f_col + m * 8 * ny * (nxh + 1)),
                     abytes + hbytes + zbytes),
        "rows_adj": (nb * (rows * f_row_r2c + box_px), zbytes + box_px * 4 + ubytes),
    }


def sectioned_work_model(pr: synth.Problem, boxes, nb: int) -> dict:
    """Algorithmic flops and bytes per launch of the sectioned kernels (PCE_FLAG_SECTIONED)
    for a chunk of nb right-hand sides, from the support boxes of w_k and the exact
    support of every h_k, with the plan's choice of sections: each term's box is cut
    into column tiles of LC - snc + 1 columns (one section each), LC the power of two
    in 16..2048 of least modelled work.  Per section: forward input window = tile
    (nr x nct), output window = tile dilated by the support (nr + snr - 1 rows,
    nct + snc - 1 columns), sections of 1024 x LC points.  Bytes: window inputs read
    once, section spectra of h read once per launch, intermediates written once and
    read once, the output window added once."""
    terms = []
    for k, (r0, nr, c0, nc) in enumerate(boxes):
        _, snr = cyclic_extent(np.any(pr.h[k] != 0, axis=1))
        _, snc = cyclic_extent(np.any(pr.h[k] != 0, axis=0))
        if nr == 0 or snr == 0:
            continue
        terms.append((nr, nc, snr, snc))
    lc = 16
    while lc < max([t[3] for t in terms] + [1]):
        lc *= 2
    best = None
    w = lc
    while w <= 2048:
        cost = sum(((nc + w - snc) // (w - snc + 1)) * ((2 * nr + snr - 1) * 2.5 * w * math.log2(w)
                                                       + (w // 2) * 2.0 * 5.0 * 1024 * 10)
                   for nr, nc, snr, snc in terms)
        if best is None or cost < best[0]:
            best = (cost, w)
        w *= 2
    lc = best[1]
    lch = lc // 2
    secs = []                                   # (in rows, in cols, out rows, out cols, term)
    for t, (nr, nc, snr, snc) in enumerate(terms):
        tw = lc - snc + 1
        for cs in range(0, nc, tw):
            nct = min(tw, nc - cs)
            secs.append((nr, nct, nr + snr - 1, nct + snc - 1, t))
    f_row = 2.5 * lc * math.log2(lc)
    f_col = 2 * 5.0 * 1024 * 10 + 6.0 * 1024        # FFT, product, inverse FFT per column
    in_rows = sum(x[0] for x in secs)
    out_rows = sum(x[2] for x in secs)
    in_px = sum(x[0] * x[1] for x in secs)
    out_px = sum(x[2] * x[3] for x in secs)
    hs = len(terms) * (lch * 1024 + 1024) * 8
    cols = len(secs) * lch
    return {
        "lc": lc, "sections": len(secs),
        "rows_r2c_window": (nb * (in_rows * f_row + in_px), nb * in_px * 4 + in_px * 4 + nb * in_rows * lch * 8),
        "cols_fwd": (nb * cols * f_col, nb * (in_rows + out_rows) * lch * 8 + hs),
        "rows_c2r": (nb * out_rows * f_row, nb * out_rows * lch * 8 + nb * out_px * 4),
        "rows_r2c": (nb * out_rows * f_row, nb * out_px * 4 + nb * out_rows * lch * 8),
        "cols_adj": (nb * cols * f_col, nb * (in_rows + out_rows) * lch * 8 + hs),
        "rows_adj": (nb * (in_rows * f_row + in_px), nb * in_rows * lch * 8 + in_px * 4 + nb * in_px * 4),
    }


def path_bytes(pr: synth.Problem, boxes) -> float:
    """Algorithmic HBM bytes of one forward + one adjoint apply of the batch:
    u and y (x and v) once, hhat once, w on its support box once, per direction."""
    if len(pr.shape) == 1:
        n = pr.shape[0]
        per = 2 * pr.batch * n * 4 + pr.m * (n // 2 + 1) * 8 + pr.m * n * 4
        return 2 * per
    ny, nx = pr.shape
    per = 2 * pr.batch * ny * nx * 4 + pr.m * ny * (nx // 2 + 1) * 8 + sum(b[1] * b[3] for b in boxes) * 4
    return 2 * per


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows: list[list[str]] = []
        self.stamps: list[float] = []
        self.t_start = 0.0
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # let nvidia-smi start sampling before the timed region begins
            t0 = time.perf_counter()
            while not self.rows and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.02)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.stamps.append(time.perf_counter())
                self.rows.append(parts)

    def mark(self):
        """Start of the timed region: samples before it (idle clocks) are not summarised."""
        self.t_start = time.perf_counter()

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self) -> dict:
        rows = [r for r, t in zip(self.rows, self.stamps) if t >= self.t_start]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.rows = rows
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            pass
    return {}


# ----------------------------------------------------------------- CPU oracle

def oracle_sample_rate(pr: synth.Problem, target_s: float = 12.0, seed: int = 5) -> dict:
    """Time the FP64 oracle (gather form) on sampled outputs of right-hand side 0.

    Returns applies/s extrapolated from the fraction of outputs computed: one
    forward and one adjoint output per sampled pixel; P sampled outputs of
    one direction count as one apply.
    """
    from oracle import expansion as E
    P = int(np.prod(pr.shape))
    rng = np.random.default_rng(seed)
    u0 = pr.u[:1]

    kept = {}

    def run(count):
        pts = np.stack([rng.integers(0, n, count) for n in pr.shape], axis=-1)
        ys, xs = [], []
        t0 = time.perf_counter()
        for i in range(0, count, 1024):          # bounded gather arrays
            ys.append(E.apply_at(u0, pr.w, pr.h, pts[i:i + 1024]))
            xs.append(E.apply_adjoint_at(u0, pr.w, pr.h, pts[i:i + 1024]))
        dt = time.perf_counter() - t0
        kept.update(pts=pts, y=np.concatenate(ys, axis=1)[0], x=np.concatenate(xs, axis=1)[0])
        return dt

    count = 16
    dt = run(count)
    while dt < 0.5 and count < P:
        count = min(P, count * 4)
        dt = run(count)
    total_pts, total_t = 0, 0.0
    while total_t < target_s and total_pts < P:
        c = int(min(P, max(count, count * (target_s - total_t) / max(dt, 1e-9) / 2)))
        t = run(c)
        total_pts += c
        total_t += t
    applies = 2.0 * total_pts / P
    return {"value": applies / total_t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{total_pts} sampled output pixels x (forward + adjoint) of right-hand side 0 "
                      f"of {pr.name}, FP64 gather form, {total_t:.1f} s",
            "seconds": total_t, "points": kept.get("pts"), "oracle_y": kept.get("y"), "oracle_x": kept.get("x")}


def reference_arm(args, pr: synth.Problem, rank: int) -> None:
    if rank != 0:
        return
    steps = []
    for _ in range(args.warmup):
        oracle_sample_rate(pr, target_s=min(2.0, args.ref_seconds), seed=1)
    last = None
    per_step = max(1.0, min(args.ref_seconds, 150.0 / max(1, args.steps)))
    for s in range(args.steps):
        last = oracle_sample_rate(pr, target_s=per_step, seed=100 + s)
        steps.append(last)
    value = statistics.median([s["value"] for s in steps])
    ms_per_step = 1000.0 * 2 * pr.batch / value
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": pr.name},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1,
                         "sample": last["sample"] if last else ""},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reference_mix_arm(args) -> None:
    """The oracle on the uneven batch: each step a bounded sample over all operators."""
    mx = synth.batch_mix(256, 4)
    steps = []
    last = None
    per_step = max(1.0, min(args.ref_seconds, 150.0 / max(1, args.steps)))
    for s in range(args.steps):
        last = oracle_mix_rate(mx, target_s=per_step, seed=100 + s)
        steps.append(last["value"])
    value = statistics.median(steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * len(mx.op_of) / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": mx.name},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1,
                         "sample": last["sample"] if last else ""},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ rank combining

def max_over_ranks(value_ms: float, dist=None, device=None) -> float:
    """Max of a per-rank time over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value_ms)
    import torch
    t = torch.tensor([float(value_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(batch_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job applies/s: every rank applies forward + adjoint to its own batch each
    step; the job takes the slowest rank's time."""
    return 2.0 * batch_per_rank * steps * world / (max_ms / 1000.0)


# ------------------------------------------------------------------- GPU arm

def gpu_arm(args, pr: synth.Problem, rank: int, world: int) -> None:
    import torch
    from paper_1604_04374_gb300 import Plan, build
    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w = torch.from_numpy(pr.w).to(dev)
    h = torch.from_numpy(pr.h).to(dev)
    u = torch.from_numpy(pr.u).to(dev)
    windows = "dense (pce_plan_create)"
    plan = None
    slots = None
    from paper_1604_04374_gb300.pce import PCE_FLAG_LOWP_STORAGE, PCE_FLAG_SECTIONED
    pflags = PCE_FLAG_LOWP_STORAGE if args.lowp else 0
    sectioned_plan = args.plan == "sectioned" and len(pr.shape) == 2
    if sectioned_plan:
        plan = Plan(w, h=h, flags=PCE_FLAG_SECTIONED | pflags)
        windows = "dense, sectioned (PCE_FLAG_SECTIONED: 1024-row sections per column tile of every box)"
    if plan is None and len(pr.shape) == 2 and "grid" in pr.meta:
        # the node-grid hats are tensor products: give the plan their factors
        wy_np, wx_np = synth.hat_factors_2d(pr.shape[0], pr.shape[1], *pr.meta["grid"])
        if np.array_equal(np.einsum("kr,kc->krc", wy_np, wx_np), pr.w):
            plan = Plan(wy=torch.from_numpy(wy_np).to(dev), wx=torch.from_numpy(wx_np).to(dev), h=h,
                        flags=pflags)
            windows = f"tensor-product hats (pce_plan_create_separable, {plan.slots()} column-factor slots)"
            if plan.slots():
                slots = slot_boxes(wy_np, wx_np)
    if plan is None:
        plan = Plan(w, h=h, flags=pflags)
    tuning = None
    if args.autotune:
        chunk, variant, rvariant, ms = plan.autotune(pr.batch, args.tuning_cache)
        tuning = {"chunk": chunk, "column_variant": variant, "row_variant": rvariant, "ms_per_apply": ms,
                  "candidates": plan.tuning_log()}
    m, boxes, scratch = plan.info()
    del w, h
    y = torch.empty_like(u)
    x = torch.empty_like(u)
    B = pr.batch
    P = int(np.prod(pr.shape))
    # L2 flush buffer (larger than the 129 MB L2), written between timed steps
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    from paper_1604_04374_gb300 import Batch

    def timed_steps(fn, sample_clocks=False, on_start=None):
        """W untimed steps, then K steps each bracketed by CUDA events on the launching
        stream (L2 flushed before each, outside the events); max over ranks of the sum."""
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        if on_start:
            on_start()
        st = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        smp = ClockSampler(torch.cuda.current_device()) if (sample_clocks and rank == 0) else None
        if smp:
            smp.__enter__()
            smp.mark()
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            st[i].record(stream)
            fn()
            en[i].record(stream)
        torch.cuda.synchronize()
        wall_s = time.perf_counter() - t0
        if smp:
            smp.__exit__(None, None, None)
        ms = max_over_ranks(sum(a_.elapsed_time(b_) for a_, b_ in zip(st, en)), dist, dev)
        return ms, wall_s, smp

    # headline step: forward and adjoint of the batch as one CUDA-graph launch of a
    # two-lane pce_batch (the two directions run concurrently, each on its own scratch)
    pair = Batch([(plan, u, y, False), (plan, u, x, True)], lanes=2)
    dev_ms, wall, sampler = timed_steps(pair.launch, sample_clocks=True)

    # the same step as two plain calls, with the library's per-kernel events
    def step():
        plan.apply(u, out=y)
        plan.apply_adjoint(u, out=x)

    seq_ms, _, _ = timed_steps(step, on_start=lambda: plan.set_timing(True))
    kern = plan.timing()
    plan.set_timing(False)
    y_ref, x_ref = y.clone(), x.clone()
    if dist:
        dist.barrier()
    launches_per_step = plan.launch_count(False, B) + plan.launch_count(True, B)

    # comparator: the plain unfused FP32 per-term pipeline on the same inputs
    comparator = None
    if args.comparator:
        from paper_1604_04374_gb300.pce import PCE_FLAG_UNFUSED
        plain = Plan(torch.from_numpy(pr.w).to(dev), h=torch.from_numpy(pr.h).to(dev), flags=PCE_FLAG_UNFUSED)

        def plain_step():
            plain.apply(u, out=y)
            plain.apply_adjoint(u, out=x)

        cms, _, _ = timed_steps(plain_step)
        comparator = {"impl": "plain unfused FP32 per-term pipeline (PCE_FLAG_UNFUSED), same FFT core",
                      "value": weak_scaling_value(B, args.steps, world, cms), "unit": UNIT,
                      "ms_per_step": cms / args.steps,
                      "launches_per_step": plain.launch_count(False, B) + plain.launch_count(True, B)}
        plain.close()

    # sectioned applies (Lemma 3.2): the same operator on per-term sections, same step
    sectioned = None
    if args.sectioned and len(pr.shape) == 2:
        from paper_1604_04374_gb300.pce import PCE_FLAG_SECTIONED, PceError
        try:
            sp = Plan(torch.from_numpy(pr.w).to(dev), h=torch.from_numpy(pr.h).to(dev),
                      flags=PCE_FLAG_SECTIONED | pflags)
        except PceError as exc:
            sectioned = {"unsupported": str(exc)}
        else:
            ys, xs = torch.empty_like(u), torch.empty_like(u)
            spair = Batch([(sp, u, ys, False), (sp, u, xs, True)], lanes=2)
            sms, _, _ = timed_steps(spair.launch)
            spair.close()

            def sstep():
                sp.apply(u, out=ys)
                sp.apply_adjoint(u, out=xs)

            sseq, _, _ = timed_steps(sstep, on_start=lambda: sp.set_timing(True))
            skern = sp.timing()
            sp.set_timing(False)

            def rel_t(a, b):
                a, b = a.reshape(B, -1).double(), b.reshape(B, -1).double()
                return float(((a - b).norm(dim=1) / b.norm(dim=1)).max())

            sectioned = {"impl": "PCE_FLAG_SECTIONED: every term on a 1024-row section, overlap-add",
                         "storage": ("half2 section spectra with per-term scale, bf16 windows" if args.lowp
                                     else "f32"),
                         "value": weak_scaling_value(B, args.steps, world, sms), "unit": UNIT,
                         "ms_per_step": sms / args.steps,
                         "launches_per_step": sp.launch_count(False, B) + sp.launch_count(True, B),
                         "max_rel_diff_vs_headline_plan": max(rel_t(ys, y_ref), rel_t(xs, x_ref)),
                         "sequential_ms_per_step": sseq / args.steps,
                         "kernel_times": skern, "chunk": plan_chunk(sp, B), "boxes": sp.info()[1]}
            sp.close()
            del ys, xs

    # gradients (pce_backward: dL/du, dL/dw, dL/dhhat of L = <H_m u, r>) per step
    backward = None
    if args.backward:
        r_t = torch.from_numpy(synth.draw(synth.rng_for(99), pr.u.shape, "normal")).to(dev)
        bms, _, _ = timed_steps(lambda: plan.backward(u, r_t))
        backward = {"value": weak_scaling_value(B / 2, args.steps, world, bms), "unit": "right-hand sides/s",
                    "ms_per_step": bms / args.steps,
                    "what": "pce_backward: dL/du (adjoint apply), dL/dw and dL/dhhat for the batch"}

    # end to end through the public API, pipelined like a serving loop: two buffer
    # sets, each bound to its own two-lane batch; step i copies its input from
    # pinned host memory (copy-in stream), runs its graph (compute stream) and
    # copies both results back (copy-out stream), overlapping step i-1 and i+1.
    pair.close()
    sets = []
    for _ in range(2):
        ud_, yd_, xd_ = torch.empty_like(u), torch.empty_like(u), torch.empty_like(u)
        sets.append((ud_, yd_, xd_, Batch([(plan, ud_, yd_, False), (plan, ud_, xd_, True)], lanes=2)))
    u_host = torch.from_numpy(pr.u).pin_memory()
    y_host = [torch.empty_like(u_host).pin_memory() for _ in range(2)]
    x_host = [torch.empty_like(u_host).pin_memory() for _ in range(2)]
    s_in, s_comp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = {key: [torch.cuda.Event() for _ in range(2)] for key in ("in", "comp", "out")}
    started = [False, False]

    def e2e_step(i):
        k = i % 2
        ud_, yd_, xd_, bt = sets[k]
        with torch.cuda.stream(s_in):
            if started[k]:
                s_in.wait_event(ev["comp"][k])      # step i-2 has consumed this input buffer
            ud_.copy_(u_host, non_blocking=True)
            ev["in"][k].record(s_in)
        with torch.cuda.stream(s_comp):
            s_comp.wait_event(ev["in"][k])
            if started[k]:
                s_comp.wait_event(ev["out"][k])     # step i-2's results have been read back
            bt.launch(s_comp)
            ev["comp"][k].record(s_comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev["comp"][k])
            y_host[k].copy_(yd_, non_blocking=True)
            x_host[k].copy_(xd_, non_blocking=True)
            ev["out"][k].record(s_out)
        started[k] = True

    for i in range(max(2, args.warmup)):
        e2e_step(i)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_in.wait_stream(stream)
    for i in range(args.steps):
        e2e_step(i)
    stream.wait_stream(s_out)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    ey, ex = y_host[(args.steps - 1) % 2], x_host[(args.steps - 1) % 2]
    if sectioned_plan:
        # sections are added with atomics: the last bits vary from run to run
        e2e_diff = max(float((ey - y_ref.cpu()).norm() / y_ref.cpu().norm()),
                       float((ex - x_ref.cpu()).norm() / x_ref.cpu().norm()))
        ok = e2e_diff < 1e-6
    else:
        ok = bool(torch.equal(ey, y_ref.cpu()) and torch.equal(ex, x_ref.cpu()))
    for st_ in sets:
        st_[3].close()

    if rank == 0:
        value = weak_scaling_value(B, args.steps, world, dev_ms)
        e2e_value = weak_scaling_value(B, args.steps, world, e2e_ms)
        clocks = sampler.summary() if sampler else {}
        sm_max = clocks.get("sm_max_mhz") or 2070.0
        # FP32 ALU peak from unit counts and clock: SMs x 128 lanes x 2 (FMA) x max SM clock
        props = torch.cuda.get_device_properties(dev)
        sms = getattr(props, "multi_processor_count", SM_COUNT_NOMINAL)
        fp32_peak_tflops = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        peaks = measured_peaks()
        hbm_peak = peaks.get("hbm_gbs")
        hbm_src = "measured" if hbm_peak else "fallback"
        hbm_peak = hbm_peak or 6800.0
        chunk = plan_chunk(plan, B)
        model = sectioned_work_model(pr, boxes, chunk) if sectioned_plan else work_model(pr, boxes, chunk, slots)
        kernels, dom = kernel_table(kern, model)
        if sectioned and "kernel_times" in sectioned:
            smodel = sectioned_work_model(pr, sectioned.pop("boxes"), sectioned["chunk"])
            sectioned["lc"] = smodel["lc"]
            sectioned["sections"] = smodel["sections"]
            sk, sdom = kernel_table(sectioned.pop("kernel_times"), smodel)
            sectioned["kernels"] = sk
            if sdom:
                sectioned["roofline"] = {
                    "kernel": sdom, "bound": "alu", "achieved": sk[sdom]["tflops"], "peak": fp32_peak_tflops,
                    "unit": "TFLOP/s", "frac": sk[sdom]["tflops"] / fp32_peak_tflops,
                    "hbm_gbs": sk[sdom]["gbs"], "hbm_frac_of_" + hbm_src: sk[sdom]["gbs"] / hbm_peak}
        roof = None
        if dom:
            d = kernels[dom]
            roof = {"kernel": dom, "bound": "alu", "achieved": d["tflops"], "peak": fp32_peak_tflops,
                    "unit": "TFLOP/s", "frac": d["tflops"] / fp32_peak_tflops,
                    "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz",
                    "traffic": MEASURED_TRAFFIC.get((pr.name, "separable" if slots else "dense", dom))
                    if (chunk == 8 and not args.lowp) else None,
                    "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch "
                                      "(profiles/kw_cols_2d_1024_m16_b8.md)",
                    "hbm_gbs": d["gbs"], "hbm_frac_of_" + hbm_src: d["gbs"] / hbm_peak}
        pbytes = path_bytes(pr, boxes)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "storage": "bf16 windows, fp16 spectra with per-term scale" if args.lowp else "f32",
            "config": {"workload": pr.name, "shape": list(pr.shape), "m": pr.m, "batch_per_gpu": B,
                       "windows": windows,
                       "global_batch": B * world, "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MB write, outside the step events)",
                       "step": "forward + adjoint apply of the batch, as one CUDA-graph launch "
                               "of a two-lane pce_batch"},
            "roofline": roof,
            "path_hbm": {"algorithmic_bytes_per_step": pbytes,
                         "gbs": pbytes * args.steps / (dev_ms / 1000.0) / 1e9,
                         "peak_gbs": hbm_peak, "peak_source": hbm_src,
                         "frac": pbytes * args.steps / (dev_ms / 1000.0) / 1e9 / hbm_peak},
            "kernels": kernels,
            "comparator": dict(comparator, speedup=value / comparator["value"]) if comparator else None,
            "sequential": {"value": weak_scaling_value(B, args.steps, world, seq_ms), "unit": UNIT,
                           "ms_per_step": seq_ms / args.steps,
                           "how": "pce_apply then pce_apply_adjoint on one stream; the per-kernel "
                                  "times and the roofline come from this pass"},
            "tuning": tuning,
            "backward": backward,
            "sectioned": sectioned,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": B * P * 4,
                    "d2h_bytes_per_step": 2 * B * P * 4,
                    "how": "pinned host u -> device, graph (forward + adjoint), both results -> pinned host, "
                           "every step; two buffer sets on copy-in / compute / copy-out streams, so copies "
                           "overlap the neighbouring steps' compute",
                    "results_match_device_run": ok,
                    "match": ("relative l2 < 1e-6 (atomic adds of the sections)" if sectioned_plan
                              else "bitwise")},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "wall_s": wall,
            "scratch_bytes": scratch,
        }
        if args.cpu_baseline and world >= 1:
            cb = oracle_sample_rate(pr, args.ref_seconds)
            line["cpu_baseline"] = {k: v for k, v in cb.items()
                                    if k not in ("seconds", "points", "oracle_y", "oracle_x")}
            # the same oracle outputs give the accuracy of this run (right-hand side 0)
            if cb.get("points") is not None:
                pts = cb["points"]
                flat = np.ravel_multi_index(tuple(pts.T), pr.shape)
                gy = y_ref[0].reshape(-1)[torch.from_numpy(flat).to(dev)].double().cpu().numpy()
                gx = x_ref[0].reshape(-1)[torch.from_numpy(flat).to(dev)].double().cpu().numpy()
                line["accuracy"] = {
                    "rel_l2_forward": float(np.linalg.norm(gy - cb["oracle_y"]) / np.linalg.norm(cb["oracle_y"])),
                    "rel_l2_adjoint": float(np.linalg.norm(gx - cb["oracle_x"]) / np.linalg.norm(cb["oracle_x"])),
                    "points": int(len(flat)), "bar": 3e-3 if args.lowp else 1e-5,
                    "against": "FP64 oracle (gather form) at the cpu_baseline leg's sampled outputs, "
                               "right-hand side 0"}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------ uneven batches

BATCH_WORKLOAD = "batch256_mixed"


def task_flops(shape, m, boxes) -> float:
    """Algorithmic FP32 flops of one apply of one right-hand side (the work model above)."""
    if len(shape) == 1:
        n = shape[0]
        fft_r = 2.5 * n * math.log2(n)
        return m * (fft_r + n + 8 * (n // 2 + 1)) + fft_r
    ny, nx = shape
    rows = sum(b[1] for b in boxes)
    box_px = sum(b[1] * b[3] for b in boxes)
    nxh1 = nx // 2 + 1
    return (rows * 2.5 * nx * math.log2(nx) + box_px + (m + 1) * nxh1 * 5.0 * ny * math.log2(ny)
            + 8.0 * m * ny * nxh1 + ny * 2.5 * nx * math.log2(nx))


def task_bytes(shape, m, boxes) -> float:
    """Algorithmic HBM bytes of one apply of one right-hand side: in, out, hhat, w on its box."""
    P = int(np.prod(shape))
    if len(shape) == 1:
        return 2 * P * 4 + m * (shape[0] // 2 + 1) * 8 + m * P * 4
    ny, nx = shape
    return 2 * P * 4 + m * ny * (nx // 2 + 1) * 8 + sum(b[1] * b[3] for b in boxes) * 4


def oracle_mix_rate(mx, target_s: float = 12.0, seed: int = 5) -> dict:
    """FP64 oracle (gather form) timed on sampled outputs of every operator of the mix
    in both directions; the whole mix's CPU time is extrapolated from the seconds
    per output of each (operator, direction)."""
    from oracle import expansion as E
    rng = np.random.default_rng(seed)
    per_op = max(0.05, target_s / (2 * len(mx.ops)))
    sec_per_out = {}
    sampled = 0
    spent = 0.0
    for oi, (shape, m, w, h) in enumerate(mx.ops):
        u0 = mx.inputs[mx.op_of.index(oi)]
        for adj in (False, True):
            fn = E.apply_adjoint_at if adj else E.apply_at
            count, dt = 8, 0.0
            while True:
                pts = np.stack([rng.integers(0, n, count) for n in shape], axis=-1)
                t0 = time.perf_counter()
                fn(u0, w, h, pts)
                dt = time.perf_counter() - t0
                if dt >= per_op or count >= int(np.prod(shape)):
                    break
                count = min(int(np.prod(shape)), count * 4)
            sec_per_out[(oi, adj)] = dt / count
            sampled += count
            spent += dt
    total = sum(int(np.prod(mx.ops[o][0])) * sec_per_out[(o, a)] for o, a in zip(mx.op_of, mx.adjoint))
    return {"value": len(mx.op_of) / total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sampled} sampled outputs over the {len(mx.ops)} operators x 2 directions of "
                      f"{mx.name}, FP64 gather form, {spent:.1f} s; whole mix extrapolated per task",
            "seconds": spent}


def batch_arm(args, rank: int, world: int) -> None:
    """256 uneven tasks (1D 4096/16384/65536, 2D 256^2/512^2/1024^2; m in 4..32;
    forward or adjoint) per step: one CUDA-graph launch of a lane-scheduled batch."""
    import torch
    from paper_1604_04374_gb300 import Batch, Plan, build
    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    mx = synth.batch_mix(256, 4)
    def make_plan(shape, m, w, h):
        """Node-grid hats are tensor products: a separable plan when the factors
        reproduce w exactly (the row transforms are shared per column factor)."""
        hd = torch.from_numpy(h).to(dev)
        if len(shape) == 2:
            wy, wx = synth.hat_factors_2d(shape[0], shape[1], *synth.node_grid(m))
            if np.array_equal(np.einsum("kr,kc->krc", wy, wx), w):
                return Plan(wy=torch.from_numpy(wy).to(dev), wx=torch.from_numpy(wx).to(dev), h=hd), True
        return Plan(torch.from_numpy(w).to(dev), h=hd), False

    made = [make_plan(*op) for op in mx.ops]
    plans = [p for p, _ in made]
    n_separable = sum(1 for _, sep in made if sep)
    tuned = []
    if args.tune_plans:
        for p in plans:
            tuned.append(p.autotune(1))
    ins = [torch.from_numpy(u).to(dev) for u in mx.inputs]
    outs = [torch.empty_like(x) for x in ins]
    tasks = [(plans[mx.op_of[i]], ins[i], outs[i], mx.adjoint[i]) for i in range(len(ins))]
    batch = Batch(tasks, lanes=args.lanes)
    batch_tuning = None
    if args.autotune:
        (cp, rp), log = batch.autotune()
        batch_tuning = {"column_policy": cp, "row_policy": rp,
                        "policies_ms_per_run": [list(t) for t in log],
                        "policy_meaning": "-1: every plan's own variant; 0/1: that variant for all tasks"}
    lanes, scratch, launches, makespan, _ = batch.info()
    n_tasks = len(tasks)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    boxes = [p.info()[1] for p in plans]
    flops = sum(task_flops(mx.ops[o][0], mx.ops[o][1], boxes[o]) for o in mx.op_of)
    nbytes = sum(task_bytes(mx.ops[o][0], mx.ops[o][1], boxes[o]) for o in mx.op_of)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(steps):
            flush.zero_()
            st[i].record(stream)
            fn()
            en[i].record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(st, en)), dist, dev)

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.__enter__()
        sampler.mark()
    graph_ms = timed(batch.launch, args.steps)
    if sampler:
        sampler.__exit__(None, None, None)
    eager_ms = timed(batch.run, args.steps)

    def sequential():
        for p, x, y, adj in tasks:
            if adj:
                p.apply_adjoint(x, out=y)
            else:
                p.apply(x, out=y)

    seq_ms = timed(sequential, args.steps) if args.comparator else None

    # end to end: every task's input from pinned host memory, the graph, every output
    # back, pipelined like a serving loop: two buffer sets, each bound to its own batch;
    # step i copies its inputs in (copy-in stream), runs its graph (compute stream) and
    # copies its outputs back (copy-out stream), overlapping steps i-1 and i+1
    ref_outs = [o.clone() for o in outs]
    hin = [torch.from_numpy(u).pin_memory() for u in mx.inputs]
    hout = [[torch.empty_like(x).pin_memory() for x in hin] for _ in range(2)]
    sets = [(ins, outs, batch)]
    ins2 = [torch.empty_like(x) for x in ins]
    outs2 = [torch.empty_like(x) for x in outs]
    tasks2 = [(plans[mx.op_of[i]], ins2[i], outs2[i], mx.adjoint[i]) for i in range(len(ins))]
    batch2 = Batch(tasks2, lanes=args.lanes)
    if args.autotune:
        batch2.autotune()
    sets.append((ins2, outs2, batch2))
    s_in, s_comp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = {key: [torch.cuda.Event() for _ in range(2)] for key in ("in", "comp", "out")}
    started = [False, False]

    def e2e_step(i):
        k = i % 2
        din, dout, bt = sets[k]
        with torch.cuda.stream(s_in):
            if started[k]:
                s_in.wait_event(ev["comp"][k])      # step i-2 has consumed these inputs
            for a, b in zip(din, hin):
                a.copy_(b, non_blocking=True)
            ev["in"][k].record(s_in)
        with torch.cuda.stream(s_comp):
            s_comp.wait_event(ev["in"][k])
            if started[k]:
                s_comp.wait_event(ev["out"][k])     # step i-2's outputs have been read back
            bt.launch(s_comp)
            ev["comp"][k].record(s_comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev["comp"][k])
            for a, b in zip(hout[k], dout):
                a.copy_(b, non_blocking=True)
            ev["out"][k].record(s_out)
        started[k] = True

    e2e_steps = max(10, args.steps // 4)
    for i in range(max(2, args.warmup)):
        e2e_step(i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_in.wait_stream(stream)
    for i in range(e2e_steps):
        e2e_step(i)
    stream.wait_stream(s_out)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    last = hout[(e2e_steps - 1) % 2]
    e2e_ok = all(torch.equal(a, b.cpu()) for a, b in zip(last, ref_outs))
    batch2.close()
    if rank == 0:
        clocks = sampler.summary() if sampler else {}
        sm_max = clocks.get("sm_max_mhz") or 2070.0
        props = torch.cuda.get_device_properties(dev)
        sms = getattr(props, "multi_processor_count", SM_COUNT_NOMINAL)
        fp32_peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        peaks = measured_peaks()
        hbm_peak = peaks.get("hbm_gbs")
        hbm_src = "measured" if hbm_peak else "fallback"
        hbm_peak = hbm_peak or 6800.0
        step_s = graph_ms / args.steps / 1000.0
        achieved = flops / step_s / 1e12
        io_bytes = sum(x.numel() * 4 for x in hin)
        line = {
            "metric": METRIC, "value": weak_scaling_value(n_tasks / 2, args.steps, world, graph_ms),
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": graph_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": mx.name, "tasks": n_tasks, "operators": len(mx.ops),
                       "shapes": [list(s) for s in synth.BATCH_SHAPES], "m": list(synth.BATCH_M),
                       "batch_per_task": 1, "lanes": lanes, "plans_autotuned": bool(args.tune_plans),
                       "windows": f"{n_separable} of {len(plans)} operators as separable plans "
                                  "(pce_plan_create_separable: 2D node-grid hats), the rest dense",
                       "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MB write, outside the step events)",
                       "step": "all tasks (forward or adjoint each) as one CUDA-graph launch"},
            "roofline": {"kernel": "whole batch", "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz",
                         "traffic": None},
            "path_hbm": {"algorithmic_bytes_per_step": nbytes, "gbs": nbytes / step_s / 1e9,
                         "peak_gbs": hbm_peak, "peak_source": hbm_src,
                         "frac": nbytes / step_s / 1e9 / hbm_peak},
            "eager_lanes": {"value": weak_scaling_value(n_tasks / 2, args.steps, world, eager_ms),
                            "ms_per_step": eager_ms / args.steps},
            "comparator": ({"impl": "the same tasks issued one by one (pce_apply / pce_apply_adjoint) "
                                    "on one stream, no lanes, no graph",
                            "value": weak_scaling_value(n_tasks / 2, args.steps, world, seq_ms),
                            "unit": UNIT, "ms_per_step": seq_ms / args.steps,
                            "speedup": seq_ms / graph_ms} if seq_ms else None),
            "e2e": {"value": weak_scaling_value(n_tasks / 2, e2e_steps, world, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
                    "how": "pinned host inputs -> device, graph, every output -> pinned host, every step; "
                           "two buffer sets on copy-in / compute / copy-out streams",
                    "results_match_device_run": e2e_ok},
            "gpu_launches": launches * args.steps,
            "clocks": clocks,
            "scratch_bytes": scratch,
            "model_makespan_ms": makespan,
            "tuning": tuned or None,
            "batch_tuning": batch_tuning,
        }
        if args.cpu_baseline:
            line["cpu_baseline"] = {k: v for k, v in oracle_mix_rate(mx, args.ref_seconds).items()
                                    if k != "seconds"}
        print(json.dumps(line), flush=True)
    batch.close()
    for p in plans:
        p.close()
    if dist:
        dist.destroy_process_group()


def kernel_table(kern: dict, model: dict):
    """Per kernel kind: launches, average time, share of the summed kernel time, and the
    work model's FP32 rate and HBM rate; with the kind of the largest share."""
    kernels = {}
    for name, (ms, n) in kern.items():
        fl, by = model.get(name, (0.0, 0.0))
        avg = ms / n
        kernels[name] = {"launches": n, "avg_us": 1000.0 * avg, "share": None,
                         "tflops": fl / (avg / 1000.0) / 1e12 if fl else None,
                         "gbs": by / (avg / 1000.0) / 1e9 if by else None}
    tot = sum(v["avg_us"] * v["launches"] for v in kernels.values()) or 1.0
    for v in kernels.values():
        v["share"] = v["avg_us"] * v["launches"] / tot
    dom = max(kernels, key=lambda k: kernels[k]["share"]) if kernels else None
    return kernels, dom


def plan_chunk(plan, batch: int) -> int:
    """Right-hand sides per launch: batch / launches-per-direction (2D), batch (1D)."""
    n = plan.launch_count(False, batch)
    per = 3 if (len(plan.shape) == 2 or plan.shape[0] > 8192) else 1
    chunks = max(1, n // per)
    return math.ceil(batch / chunks)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="2d_1024_m16_b8", choices=sorted(synth.WORKLOADS) + [BATCH_WORKLOAD])
    ap.add_argument("--lanes", type=int, default=16, help="streams of the uneven batch")
    ap.add_argument("--autotune", dest="autotune", action="store_true", default=True,
                    help="autotune the plan(s) before timing (default)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--backward", action="store_true", help="also time pce_backward (gradients)")
    ap.add_argument("--plan", default="auto", choices=["auto", "sectioned"],
                    help="headline plan: auto (separable for node-grid hats, else dense) or sectioned")
    ap.add_argument("--sectioned", action="store_true",
                    help="also time the same step with a sectioned plan (PCE_FLAG_SECTIONED)")
    ap.add_argument("--lowp", action="store_true",
                    help="reduced storage (PCE_FLAG_LOWP_STORAGE: bf16 windows, fp16 spectra)")
    ap.add_argument("--tuning-cache", default=None,
                    help="JSON-lines autotuner cache: reuse earlier choices instead of timing again")
    ap.add_argument("--tune-plans", action="store_true",
                    help="uneven batch: autotune every plan in isolation first")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-comparator", dest="comparator", action="store_false")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == BATCH_WORKLOAD:
        if args.impl == "reference":
            if rank == 0:
                reference_mix_arm(args)
            return
        batch_arm(args, rank, world)
        return
    pr = synth.workload(args.workload)
    if args.impl == "reference":
        reference_arm(args, pr, rank)
        return
    gpu_arm(args, pr, rank, world)


if __name__ == "__main__":
    main()
