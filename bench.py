"""Benchmark of the convolution-product expansion apply (Eq. 1.4) and its adjoint.

One step = one forward apply y = H_m u and one adjoint apply x = H_m^* u of a
whole batch of right-hand sides (every kernel of the hot path runs once per
chunk of the batch).  Metric: applies per second, counting each right-hand
side of each direction as one apply.

Headline workload: 2D periodic 1024 x 1024 float32 images, batch 8, m = 16
bilinear hat windows on a 4 x 4 node grid, anisotropic rotated Gaussian PSFs
(sigma_x = 1.5 + y1, sigma_y = 1.5 + y2 px, theta = pi y1 y2), u ~ U[0,1).
The default run then measures every other workload of the benchmark set under
"configs": 1D N = 1024 (m = 8, B = 1); 2D 512^2 (m = 16, B = 16) with the
gradients; 2D 2048^2 (m = 64, B = 4) whole-grid and sectioned, each with FP32
and reduced (bf16 w / fp16 hhat) storage; and 256 uneven tasks in one graph.
Each carries its own clock samples, accuracy against the FP64 oracle,
roofline and end-to-end figures.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Under torchrun (N > 1) every rank runs its own batch (weak scaling: the
right-hand sides are independent, no data-path collective), the step time is
the max over ranks and rank 0 prints the JSON line.  ``--impl reference``
times the compiled FP64 CPU oracle on the host cores: each step is the
forward and the adjoint apply of one right-hand side of the same workload,
every output computed.
"""
from __future__ import annotations

import argparse
import copy
import json
import math
import os
import platform
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
HEADLINE = "2d_1024_m16_b8"
BATCH_WORKLOAD = "batch256_mixed"
# the other workloads of the default run: (name, workload, option overrides)
SUB_CONFIGS = (
    ("1d_n1024_m8_b1", "1d_n1024_m8_b1", {}),
    ("2d_512_m16_b16", "2d_512_m16_b16", {"backward": True}),
    ("2d_2048_m64_b4_whole_f32", "2d_2048_m64_b4", {}),
    ("2d_2048_m64_b4_whole_lowp", "2d_2048_m64_b4", {"lowp": True, "comparator": False}),
    ("2d_2048_m64_b4_sectioned_f32", "2d_2048_m64_b4", {"plan": "sectioned", "comparator": False}),
    ("2d_2048_m64_b4_sectioned_lowp", "2d_2048_m64_b4", {"plan": "sectioned", "lowp": True,
                                                         "comparator": False}),
    (BATCH_WORKLOAD, BATCH_WORKLOAD, {}),
)

# DRAM bytes (read + write) per launch measured by ncu, keyed by (workload,
# plan kind, kernel kind, column variant, right-hand sides per launch); valid
# only for the kernels as captured, each entry naming its profile summary.
MEASURED_TRAFFIC = {
    ("2d_1024x1024_m16_b8", "separable", "cols_fwd", 2, 8): (201.729280e6 + 21.671936e6,
                                                             "profiles/kt_cols_2d_1024_m16_b8.md"),
    ("2d_1024x1024_m16_b8", "separable", "cols_adj", 2, 8): (101.006848e6 + 89.132800e6,
                                                             "profiles/kt_cols_2d_1024_m16_b8.md"),
    ("2d_512x512_m16_b16", "separable", "cols_fwd", 2, 16): (84.358400e6 + 4.101632e6,
                                                            "profiles/kt_cols_2d_512_m16_b16.md"),
    ("2d_512x512_m16_b16", "separable", "cols_adj", 2, 16): (33.777408e6 + 18.606336e6,
                                                            "profiles/kt_cols_2d_512_m16_b16.md"),
}

# ------------------------------------------------------------- algorithmic work


def cyclic_extent(flags) -> tuple[int, int]:
    """Smallest periodic arc [start, start + n) holding every True entry: (start, n)."""
    flags = np.asarray(flags, dtype=bool)
    n = len(flags)
    if not flags.any():
        return 0, 0
    if flags.all():
        return 0, n
    idx = np.nonzero(flags)[0]
    gaps = np.diff(np.concatenate([idx, [idx[0] + n]]))
    g = int(np.argmax(gaps))
    start = int(idx[(g + 1) % len(idx)])
    return start, n - int(gaps[g]) + 1


def slot_boxes(wy: np.ndarray, wx: np.ndarray) -> list:
    """Boxes (r0, nr, c0, nc) of the slots of tensor-product windows: one slot per distinct
    column factor, rows = union of the slot's row supports, columns = the factor's support."""
    slots = {}
    for k in range(wy.shape[0]):
        key = wx[k].tobytes()
        rows = wy[k] != 0
        slots[key] = (slots[key][0] | rows, wx[k]) if key in slots else (rows, wx[k])
    out = []
    for rows, f in slots.values():
        r0, nr = cyclic_extent(rows)
        c0, nc = cyclic_extent(f != 0)
        out.append((r0, nr, c0, nc))
    return out


def work_model(pr: synth.Problem, boxes, nb: int, slots=None) -> dict:
    """Per kernel kind, for a chunk of nb right-hand sides: (algorithmic FP32 flops,
    algorithmic HBM bytes, scratch bytes).

    Flops are the nominal FFT counts (5 N log2 N per complex N-point FFT,
    2.5 N log2 N per real one), 8 per complex multiply-add, 1 per window
    multiply.  Algorithmic bytes are what the method must move: u and y once,
    hhat once, w on its support box once (the row factors once for separable
    windows).  Scratch bytes are the intermediates Z/Q and A/V, which the
    design keeps out of the algorithmic count (they would stay on chip or in
    L2 in an ideal schedule) and which are reported beside it.  With `slots`
    (separable windows) the row passes transform one row set per slot instead
    of one per term, the column passes multiply by the row factors.
    """
    if len(pr.shape) == 1:
        n = pr.shape[0]
        m = pr.m
        fft_r = 2.5 * n * math.log2(n)
        fl = nb * (m * (fft_r + n + 8 * (n // 2 + 1)) + fft_r)
        by = nb * n * 8 + m * (n // 2 + 1) * 8 + m * n * 4
        return {"fwd_1d": (fl, by, 0.0), "adj_1d": (fl, by, 0.0)}
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
        wrows = m * ny * 4
        cfl = nb * ((m + 1) * (nxh + 1) * f_col + m * 8 * ny * (nxh + 1) + rows * (nxh + 1) * 2)
        return {
            "rows_r2c_window": (nb * (srows * f_row_r2c + spx), ubytes + wcols, sbytes),
            "cols_fwd": (cfl, hbytes + wrows, sbytes + abytes),
            "rows_c2r": (nb * ny * f_row_r2c, ubytes, abytes),
            "rows_r2c": (nb * ny * f_row_r2c, ubytes, abytes),
            "cols_adj": (cfl, hbytes + wrows, abytes + sbytes),
            "rows_adj": (nb * (srows * f_row_r2c + spx), wcols + ubytes, sbytes),
        }
    return {
        "rows_r2c_window": (nb * (rows * f_row_r2c + box_px), ubytes + box_px * 4, zbytes),
        "cols_fwd": (nb * ((m + 1) * (nxh + 1) * f_col + m * 8 * ny * (nxh + 1)), hbytes, zbytes + abytes),
        "rows_c2r": (nb * ny * f_row_r2c, ubytes, abytes),
        "rows_r2c": (nb * ny * f_row_r2c, ubytes, abytes),
        "cols_adj": (nb * ((m + 1) * (nxh + 1) * f_col + m * 8 * ny * (nxh + 1)), hbytes, abytes + zbytes),
        "rows_adj": (nb * (rows * f_row_r2c + box_px), box_px * 4 + ubytes, zbytes),
    }


def sectioned_work_model(pr: synth.Problem, boxes, nb: int) -> dict:
    """Per sectioned kernel kind (PCE_FLAG_SECTIONED) and chunk of nb right-hand sides:
    (flops, algorithmic bytes, scratch bytes), from the support boxes of w_k and the
    exact support of every h_k, with the plan's choice of sections: each term's box
    is cut into column tiles of LC - snc + 1 columns (one section each), LC the power
    of two in 16..2048 of least modelled work.  Per section: forward input window =
    tile (nr x nct), output window = tile dilated by the support (nr + snr - 1 rows,
    nct + snc - 1 columns), sections of 1024 x LC points.  Algorithmic bytes: window
    inputs and outputs once, section spectra of h once, window box once; scratch:
    the section intermediates written and read once each."""
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
    zin = nb * in_rows * lch * 8
    zout = nb * out_rows * lch * 8
    return {
        "lc": lc, "sections": len(secs),
        "rows_r2c_window": (nb * (in_rows * f_row + in_px), nb * in_px * 4 + in_px * 4, zin),
        "cols_fwd": (nb * cols * f_col, hs, zin + zout),
        "rows_c2r": (nb * out_rows * f_row, nb * out_px * 4, zout),
        "rows_r2c": (nb * out_rows * f_row, nb * out_px * 4, zout),
        "cols_adj": (nb * cols * f_col, hs, zin + zout),
        "rows_adj": (nb * (in_rows * f_row + in_px), in_px * 4 + nb * in_px * 4, zin),
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
        self.t_end = None
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

    def end(self):
        """End of the timed region: keep sampling one more period (the reading of the last
        moments under load arrives after it)."""
        self.t_end = time.perf_counter()
        time.sleep(0.15)

    def __exit__(self, *exc):
        if self.t_end is None:
            self.t_end = time.perf_counter()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self) -> dict:
        hi = (self.t_end or time.perf_counter()) + 0.12
        rows = [r for r, t in zip(self.rows, self.stamps) if self.t_start <= t <= hi]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            pass
    return {}


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


# ----------------------------------------------------------------- CPU oracle

def oracle_threads_wanted() -> int:
    """The host cores this process may run on (the affinity mask)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle():
    os.environ.setdefault("OMP_NUM_THREADS", str(oracle_threads_wanted()))
    from oracle import direct
    return direct


def oracle_rhs0(pr: synth.Problem) -> dict:
    """The compiled FP64 oracle on right-hand side 0, every output of both directions,
    timed on the host cores.  Returns the outputs, the time and a cpu_baseline record."""
    C = _oracle()
    u0 = pr.u[:1]
    t0 = time.perf_counter()
    y = C.apply(u0, pr.w, pr.h)[0]
    x = C.apply_adjoint(u0, pr.w, pr.h)[0]
    dt = time.perf_counter() - t0
    return {"y": y, "x": x, "seconds": dt,
            "cpu_baseline": {"value": 2.0 / dt, "unit": UNIT, "cores": C.threads(), "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"forward + adjoint of right-hand side 0 of {pr.name}, every output, "
                                       f"FP64 direct summation (oracle/direct.c, OpenMP), {dt:.2f} s"}}


def oracle_mix_rate(mx, target_s: float = 12.0, seed: int = 5) -> dict:
    """The compiled FP64 oracle on sampled outputs of every operator of the uneven mix
    in both directions; the whole mix's CPU time is extrapolated from the seconds
    per output of each (operator, direction)."""
    C = _oracle()
    rng = np.random.default_rng(seed)
    per_op = max(0.05, target_s / (2 * len(mx.ops)))
    sec_per_out = {}
    sampled = 0
    spent = 0.0
    for oi, (shape, m, w, h) in enumerate(mx.ops):
        u0 = mx.inputs[mx.op_of.index(oi)]
        for adj in (False, True):
            fn = C.apply_adjoint_at if adj else C.apply_at
            count, dt = 64, 0.0
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
    return {"value": len(mx.op_of) / total, "unit": UNIT, "cores": C.threads(), "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{sampled} sampled outputs over the {len(mx.ops)} operators x 2 directions of "
                      f"{mx.name}, FP64 direct summation (oracle/direct.c, OpenMP), {spent:.1f} s; "
                      "whole mix extrapolated per task",
            "seconds": spent}


def headline_config(pr: synth.Problem, world: int) -> dict:
    """The config block of a plan workload, the same for the GPU and the reference arm."""
    sep = len(pr.shape) == 2 and "grid" in pr.meta
    return {"workload": pr.name, "shape": list(pr.shape), "m": pr.m, "batch_per_gpu": pr.batch,
            "global_batch": pr.batch * world, "parallelism": f"replicas x{world}",
            "windows": ("tensor-product hats on a node grid" if sep else "hats") + f", m = {pr.m}",
            "l2": "flushed between timed steps (256 MB write, outside the step events)",
            "step": "forward + adjoint apply of the batch"}


def mix_config(mx, world: int) -> dict:
    return {"workload": mx.name, "tasks": len(mx.op_of), "operators": len(mx.ops),
            "shapes": [list(s) for s in synth.BATCH_SHAPES], "m": list(synth.BATCH_M), "batch_per_task": 1,
            "parallelism": f"replicas x{world}",
            "l2": "flushed between timed steps (256 MB write, outside the step events)",
            "step": "all tasks (forward or adjoint each)"}


def reference_arm(args, workload: str, rank: int, world: int) -> None:
    """The FP64 oracle (oracle/direct.c) on the host cores.  Plan workloads: every
    step is the forward and the adjoint apply of one right-hand side, every output
    computed (2 applies per step).  The uneven mix: every step is a bounded sample
    over all operators, extrapolated per task."""
    if rank != 0:
        return
    if workload == BATCH_WORKLOAD:
        mx = synth.batch_mix(256, 4)
        per_step = max(1.0, min(args.ref_seconds, 150.0 / max(1, args.steps)))
        for s in range(args.warmup):
            oracle_mix_rate(mx, target_s=0.5, seed=1 + s)
        vals, last = [], None
        for s in range(args.steps):
            last = oracle_mix_rate(mx, target_s=per_step, seed=100 + s)
            vals.append(last["value"])
        value = statistics.median(vals)
        ms_per_step = 1000.0 * statistics.median([per_step] * args.steps)
        config = mix_config(mx, world)
        sample = last["sample"] if last else ""
        cores = last["cores"] if last else 1
    else:
        pr = synth.workload(workload)
        C = _oracle()
        u0 = pr.u[:1]

        def step():
            C.apply(u0, pr.w, pr.h)
            C.apply_adjoint(u0, pr.w, pr.h)

        for _ in range(args.warmup):
            step()
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            step()
            times.append(time.perf_counter() - t0)
        total = sum(times)
        value = 2.0 * args.steps / total
        ms_per_step = 1000.0 * total / args.steps
        config = headline_config(pr, world)
        cores = C.threads()
        sample = (f"each step: forward + adjoint of right-hand side 0 of {pr.name}, every output, "
                  "FP64 direct summation (oracle/direct.c, OpenMP)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": cores, "cpu_model": cpu_model(),
                         "sample": sample},
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

class Ctx:
    """What every measurement shares: the device, the process group, the L2 flush."""

    def __init__(self, rank: int, world: int):
        import torch
        from paper_1604_04374_gb300 import build
        build.build()
        self.torch = torch
        self.rank, self.world = rank, world
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        self.dev = torch.device("cuda", local)
        self.dist = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=self.dev)
            self.dist = dist
        # L2 flush buffer (larger than the 129 MB L2), written between timed steps
        self.flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=self.dev)
        props = torch.cuda.get_device_properties(self.dev)
        self.sms = getattr(props, "multi_processor_count", SM_COUNT_NOMINAL)
        peaks = measured_peaks()
        self.hbm_peak = peaks.get("hbm_gbs") or 6800.0
        self.hbm_src = "measured" if peaks.get("hbm_gbs") else "fallback"

    def fp32_peak(self, sm_max_mhz) -> float:
        """FP32 ALU peak from unit counts and clock: SMs x 128 lanes x 2 (FMA) x max SM clock."""
        return self.sms * FP32_LANES_PER_SM * 2 * (sm_max_mhz or 2070.0) * 1e6 / 1e12

    def peak_source(self, sm_max_mhz) -> str:
        return f"derived: {self.sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max_mhz or 2070.0:.0f} MHz"

    def timed(self, fn, steps: int, warmup: int, sample_clocks=False, on_start=None, min_seconds=0.0):
        """W untimed steps, then K steps each bracketed by CUDA events on the launching
        stream (L2 flushed before each, outside the events); max over ranks of the sum.
        min_seconds > 0 raises K until the timed region lasts about that long (the
        clock samples need a few tenths of a second).  Returns (ms, steps, wall_s, clocks)."""
        torch = self.torch
        stream = torch.cuda.current_stream()
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if min_seconds > 0:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            per = max(e0.elapsed_time(e1), 1e-3) / 1000.0
            steps = max(steps, min(100000, int(math.ceil(min_seconds / per))))
        if on_start:
            on_start()
        st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        if self.dist:
            self.dist.barrier()
        torch.cuda.synchronize()
        smp = ClockSampler(torch.cuda.current_device()) if (sample_clocks and self.rank == 0) else None
        if smp:
            smp.__enter__()
            smp.mark()
        t0 = time.perf_counter()
        for i in range(steps):
            self.flush.zero_()
            st[i].record(stream)
            fn()
            en[i].record(stream)
        torch.cuda.synchronize()
        wall_s = time.perf_counter() - t0
        clocks = None
        if smp:
            smp.end()
            smp.__exit__(None, None, None)
            clocks = smp.summary()
        ms = max_over_ranks(sum(a_.elapsed_time(b_) for a_, b_ in zip(st, en)), self.dist, self.dev)
        return ms, steps, wall_s, clocks

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()


def kernel_table(kern: dict, model: dict, hbm_peak: float, units: int | None = None):
    """Per kernel kind: launches, average time, share of the summed kernel time, the work
    model's FP32 rate, its HBM rate of algorithmic bytes (and the fraction of the HBM
    peak), and the scratch bytes per launch; with the kind of the largest share.
    `units`: how many times the model's work ran (timed steps x chunks of right-hand
    sides per step); a kind launched several times per chunk (the slot-by-slot
    schedule) is averaged per chunk, so that its rate is comparable with one launch
    of the single-pass schedule."""
    kernels = {}
    for name, (ms, n) in kern.items():
        fl, by, scr = model.get(name, (0.0, 0.0, 0.0))
        per = n // units if units and n % units == 0 and n >= units else 1
        avg = ms / (n // per)
        gbs = by / (avg / 1000.0) / 1e9 if by else None
        kernels[name] = {"launches": n, "launches_per_chunk": per, "avg_us": 1000.0 * avg, "share": None,
                         "tflops": fl / (avg / 1000.0) / 1e12 if fl else None,
                         "algorithmic_gbs": gbs, "hbm_frac": gbs / hbm_peak if gbs else None,
                         "scratch_bytes_per_launch": scr}
    tot = sum(v["avg_us"] * v["launches"] / v["launches_per_chunk"] for v in kernels.values()) or 1.0
    for v in kernels.values():
        v["share"] = v["avg_us"] * v["launches"] / v["launches_per_chunk"] / tot
    dom = max(kernels, key=lambda k: kernels[k]["share"]) if kernels else None
    return kernels, dom


def plan_chunk(plan, batch: int) -> int:
    """Right-hand sides per launch: the batch in equal chunks of at most the plan's chunk
    (pce_plan_tuning), as the library splits it."""
    chunk = max(1, plan.tuning()[0])
    nch = math.ceil(batch / chunk)
    return math.ceil(batch / nch)


def rel_l2(got: np.ndarray, ref: np.ndarray) -> float:
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def gpu_arm(args, pr: synth.Problem, ctx: Ctx, oracle_cache: dict, headline: bool) -> dict | None:
    """Measure one plan workload; returns the JSON record on rank 0."""
    torch = ctx.torch
    dev = ctx.dev
    from paper_1604_04374_gb300 import Batch, Plan
    from paper_1604_04374_gb300.pce import PCE_FLAG_LOWP_STORAGE, PCE_FLAG_SECTIONED, PCE_FLAG_UNFUSED
    world = ctx.world
    w = torch.from_numpy(pr.w).to(dev)
    h = torch.from_numpy(pr.h).to(dev)
    u = torch.from_numpy(pr.u).to(dev)
    windows = "dense (pce_plan_create)"
    plan = None
    slots = None
    kind = "dense"
    pflags = PCE_FLAG_LOWP_STORAGE if args.lowp else 0
    sectioned_plan = args.plan == "sectioned" and len(pr.shape) == 2
    if sectioned_plan:
        plan = Plan(w, h=h, flags=PCE_FLAG_SECTIONED | pflags)
        windows = "dense, sectioned (PCE_FLAG_SECTIONED: 1024-row sections per column tile of every box)"
        kind = "sectioned"
    if plan is None and len(pr.shape) == 2 and "grid" in pr.meta:
        # the node-grid hats are tensor products: give the plan their factors
        wy_np, wx_np = synth.hat_factors_2d(pr.shape[0], pr.shape[1], *pr.meta["grid"])
        if np.array_equal(np.einsum("kr,kc->krc", wy_np, wx_np), pr.w):
            plan = Plan(wy=torch.from_numpy(wy_np).to(dev), wx=torch.from_numpy(wx_np).to(dev), h=h,
                        flags=pflags)
            windows = f"tensor-product hats (pce_plan_create_separable, {plan.slots()} column-factor slots)"
            if plan.slots():
                slots = slot_boxes(wy_np, wx_np)
                kind = "separable"
    if plan is None:
        plan = Plan(w, h=h, flags=pflags)
    tuning = None
    if args.col_variant is not None:
        plan.set_tuning(0, args.col_variant, args.row_variant or 0)
        tuning = {"forced": True, "column_variant": args.col_variant, "row_variant": args.row_variant or 0}
    elif args.autotune:
        chunk, variant, rvariant, ms = plan.autotune(pr.batch, args.tuning_cache)
        tuning = {"chunk": chunk, "column_variant": variant, "row_variant": rvariant, "ms_per_apply": ms,
                  "candidates": plan.tuning_log()}
    col_variant = plan.tuning()[1]
    nb = plan_chunk(plan, pr.batch)
    m, boxes, scratch = plan.info()
    del w, h
    y = torch.empty_like(u)
    x = torch.empty_like(u)
    B = pr.batch
    P = int(np.prod(pr.shape))
    min_s = 0.0 if headline else 0.3

    # the step: forward and adjoint of the batch as one CUDA-graph launch of a
    # two-lane pce_batch (the two directions run concurrently, each on its own scratch)
    pair = Batch([(plan, u, y, False), (plan, u, x, True)], lanes=2)
    dev_ms, steps, wall, clocks = ctx.timed(pair.launch, args.steps, args.warmup, sample_clocks=True,
                                            min_seconds=min_s)

    # the same step as two plain calls, with the library's per-kernel events
    def step():
        plan.apply(u, out=y)
        plan.apply_adjoint(u, out=x)

    seq_ms, seq_steps, _, _ = ctx.timed(step, min(steps, max(args.steps, 20)), args.warmup,
                                        on_start=lambda: plan.set_timing(True))
    kern = plan.timing()
    plan.set_timing(False)
    y_ref, x_ref = y.clone(), x.clone()
    launches_per_step = plan.launch_count(False, B) + plan.launch_count(True, B)

    # comparator: the plain unfused FP32 per-term pipeline on the same inputs
    comparator = None
    if args.comparator and len(pr.shape) == 2:
        plain = Plan(torch.from_numpy(pr.w).to(dev), h=torch.from_numpy(pr.h).to(dev), flags=PCE_FLAG_UNFUSED)

        def plain_step():
            plain.apply(u, out=y)
            plain.apply_adjoint(u, out=x)

        cms, csteps, _, _ = ctx.timed(plain_step, max(3, min(args.steps, 20)), args.warmup)
        comparator = {"impl": "plain unfused FP32 per-term pipeline (PCE_FLAG_UNFUSED), same FFT core",
                      "value": weak_scaling_value(B, csteps, world, cms), "unit": UNIT,
                      "ms_per_step": cms / csteps,
                      "launches_per_step": plain.launch_count(False, B) + plain.launch_count(True, B)}
        plain.close()

    # gradients (pce_backward: dL/du, dL/dw, dL/dhhat of L = <H_m u, r>) per step
    backward = None
    if args.backward:
        r_t = torch.from_numpy(synth.draw(synth.rng_for(99), pr.u.shape, "normal")).to(dev)
        bms, bsteps, _, bclocks = ctx.timed(lambda: plan.backward(u, r_t), args.steps, args.warmup,
                                            sample_clocks=True, min_seconds=0.3)
        backward = {"value": weak_scaling_value(B / 2, bsteps, world, bms), "unit": "right-hand sides/s",
                    "ms_per_step": bms / bsteps, "steps": bsteps, "clocks": bclocks,
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

    stream = torch.cuda.current_stream()
    for i in range(max(2, args.warmup)):
        e2e_step(i)
    torch.cuda.synchronize()
    if ctx.dist:
        ctx.dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_in.wait_stream(stream)
    for i in range(steps):
        e2e_step(i)
    stream.wait_stream(s_out)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), ctx.dist, dev)
    ey, ex = y_host[(steps - 1) % 2], x_host[(steps - 1) % 2]
    if sectioned_plan:
        # sections are added with atomics: the last bits vary from run to run
        e2e_diff = max(float((ey - y_ref.cpu()).norm() / y_ref.cpu().norm()),
                       float((ex - x_ref.cpu()).norm() / x_ref.cpu().norm()))
        ok = e2e_diff < 1e-6
    else:
        ok = bool(torch.equal(ey, y_ref.cpu()) and torch.equal(ex, x_ref.cpu()))
    for st_ in sets:
        st_[3].close()
    plan.close()
    if ctx.rank != 0:
        return None

    value = weak_scaling_value(B, steps, world, dev_ms)
    e2e_value = weak_scaling_value(B, steps, world, e2e_ms)
    clocks = clocks or {}
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    fp32_peak = ctx.fp32_peak(sm_max)
    model = sectioned_work_model(pr, boxes, nb) if sectioned_plan else work_model(pr, boxes, nb, slots)
    kernels, dom = kernel_table(kern, model, ctx.hbm_peak, seq_steps * math.ceil(B / nb))
    roof = None
    if dom:
        d = kernels[dom]
        traffic = MEASURED_TRAFFIC.get((pr.name, kind, dom, col_variant, nb)) if not args.lowp else None
        roof = {"kernel": dom, "bound": "alu", "achieved": d["tflops"], "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": d["tflops"] / fp32_peak if d["tflops"] else None,
                "peak_source": ctx.peak_source(sm_max),
                "traffic": traffic[0] if traffic else None,
                "algorithmic_bytes_per_launch": model[dom][1],
                "scratch_bytes_per_launch": model[dom][2],
                "hbm_gbs": d["algorithmic_gbs"], "hbm_peak_gbs": ctx.hbm_peak, "hbm_peak_source": ctx.hbm_src,
                "hbm_frac": d["hbm_frac"]}
        if traffic:
            roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch "
                                      f"({traffic[1]})")
    pbytes = path_bytes(pr, boxes)
    rec = {
        "value": value, "unit": UNIT, "steps": steps, "ms_per_step": dev_ms / steps,
        "storage": "bf16 windows, fp16 spectra with per-term scale" if args.lowp else "f32",
        "plan": {"kind": kind, "windows": windows, "column_variant": col_variant, "right_hand_sides_per_launch": nb,
                 "boxes": len(boxes), "scratch_bytes": scratch},
        "roofline": roof,
        "path_hbm": {"algorithmic_bytes_per_step": pbytes,
                     "gbs": pbytes * steps / (dev_ms / 1000.0) / 1e9,
                     "peak_gbs": ctx.hbm_peak, "peak_source": ctx.hbm_src,
                     "frac": pbytes * steps / (dev_ms / 1000.0) / 1e9 / ctx.hbm_peak},
        "kernels": kernels,
        "comparator": dict(comparator, speedup=value / comparator["value"]) if comparator else None,
        "sequential": {"value": weak_scaling_value(B, seq_steps, world, seq_ms), "unit": UNIT,
                       "ms_per_step": seq_ms / seq_steps,
                       "how": "pce_apply then pce_apply_adjoint on one stream; the per-kernel "
                              "times and the roofline come from this pass"},
        "tuning": tuning,
        "backward": backward,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": B * P * 4,
                "d2h_bytes_per_step": 2 * B * P * 4,
                "how": "pinned host u -> device, graph (forward + adjoint), both results -> pinned host, "
                       "every step; two buffer sets on copy-in / compute / copy-out streams, so copies "
                       "overlap the neighbouring steps' compute",
                "results_match_device_run": ok,
                "match": ("relative l2 < 1e-6 (atomic adds of the sections)" if sectioned_plan
                          else "bitwise")},
        "gpu_launches": launches_per_step * steps,
        "clocks": clocks,
        "wall_s": wall,
    }
    if args.cpu_baseline:
        if pr.name not in oracle_cache:
            oracle_cache[pr.name] = oracle_rhs0(pr)
        orc = oracle_cache[pr.name]
        rec["cpu_baseline"] = orc["cpu_baseline"]
        gy = y_ref[0].double().cpu().numpy()
        gx = x_ref[0].double().cpu().numpy()
        rec["accuracy"] = {"rel_l2_forward": rel_l2(gy, orc["y"]), "rel_l2_adjoint": rel_l2(gx, orc["x"]),
                           "outputs": int(P), "bar": 3e-3 if args.lowp else 1e-5,
                           "against": "FP64 oracle (oracle/direct.c), every output of right-hand side 0"}
    return rec


def batch_arm(args, ctx: Ctx) -> dict | None:
    """256 uneven tasks (1D 4096/16384/65536, 2D 256^2/512^2/1024^2; m in 4..32;
    forward or adjoint) per step: one CUDA-graph launch of a lane-scheduled batch."""
    torch = ctx.torch
    dev = ctx.dev
    world = ctx.world
    from paper_1604_04374_gb300 import Batch, Plan
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
                        "policy_meaning": "-1: every plan's own variant; 0/1/2: that variant for every task that has it"}
    lanes, scratch, launches, makespan, _ = batch.info()
    n_tasks = len(tasks)
    boxes = [p.info()[1] for p in plans]
    flops = sum(task_flops(mx.ops[o][0], mx.ops[o][1], boxes[o]) for o in mx.op_of)
    nbytes = sum(task_bytes(mx.ops[o][0], mx.ops[o][1], boxes[o]) for o in mx.op_of)

    graph_ms, steps, wall, clocks = ctx.timed(batch.launch, args.steps, args.warmup, sample_clocks=True,
                                              min_seconds=0.3)
    eager_ms, esteps, _, _ = ctx.timed(batch.run, max(3, min(args.steps, 20)), args.warmup)

    def sequential():
        for p, x_, y_, adj in tasks:
            if adj:
                p.apply_adjoint(x_, out=y_)
            else:
                p.apply(x_, out=y_)

    seq_ms, qsteps = (None, 0)
    if args.comparator:
        seq_ms, qsteps, _, _ = ctx.timed(sequential, max(3, min(args.steps, 20)), args.warmup)

    # end to end: every task's input from pinned host memory, the graph, every output
    # back, pipelined like a serving loop: two buffer sets, each bound to its own batch;
    # step i copies its inputs in (copy-in stream), runs its graph (compute stream) and
    # copies its outputs back (copy-out stream), overlapping steps i-1 and i+1
    batch.launch()
    torch.cuda.synchronize()
    ref_outs = [o.clone() for o in outs]
    hin = [torch.from_numpy(u).pin_memory() for u in mx.inputs]
    hout = [[torch.empty_like(x).pin_memory() for x in hin] for _ in range(2)]
    sets = [(ins, outs, batch)]
    ins2 = [torch.empty_like(x) for x in ins]
    outs2 = [torch.empty_like(x) for x in outs]
    tasks2 = [(plans[mx.op_of[i]], ins2[i], outs2[i], mx.adjoint[i]) for i in range(len(ins))]
    batch2 = Batch(tasks2, lanes=args.lanes)
    if batch_tuning:   # the same policies as the measured batch: the same rounding, bitwise equal results
        batch2.set_tuning(batch_tuning["column_policy"], batch_tuning["row_policy"])
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

    stream = torch.cuda.current_stream()
    e2e_steps = max(10, min(steps, 200))
    for i in range(max(2, args.warmup)):
        e2e_step(i)
    torch.cuda.synchronize()
    if ctx.dist:
        ctx.dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_in.wait_stream(stream)
    for i in range(e2e_steps):
        e2e_step(i)
    stream.wait_stream(s_out)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), ctx.dist, dev)
    last = hout[(e2e_steps - 1) % 2]
    e2e_ok = all(torch.equal(a, b.cpu()) for a, b in zip(last, ref_outs))
    batch2.close()
    # accuracy: every output of a few tasks of each kind against the oracle
    acc = None
    if args.cpu_baseline and ctx.rank == 0:
        C = _oracle()
        worst = {}
        seen = set()
        for i in range(n_tasks):
            o = mx.op_of[i]
            key = (mx.ops[o][0], mx.adjoint[i])
            if key in seen or int(np.prod(mx.ops[o][0])) > 512 * 512:
                continue
            seen.add(key)
            shape, m_, w_, h_ = mx.ops[o]
            fn = C.apply_adjoint if mx.adjoint[i] else C.apply
            ref = fn(mx.inputs[i], w_, h_)
            got = ref_outs[i].double().cpu().numpy()
            name = "x".join(str(s) for s in shape) + (" adjoint" if mx.adjoint[i] else " forward")
            worst[name] = rel_l2(got, ref)
        acc = {"rel_l2_max": max(worst.values()) if worst else None, "per_kind": worst, "bar": 1e-5,
               "against": "FP64 oracle (oracle/direct.c), every output of the first task of each "
                          "(shape, direction) up to 512 x 512"}
    batch.close()
    for p in plans:
        p.close()
    if ctx.rank != 0:
        return None
    clocks = clocks or {}
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    fp32_peak = ctx.fp32_peak(sm_max)
    step_s = graph_ms / steps / 1000.0
    achieved = flops / step_s / 1e12
    io_bytes = sum(x.numel() * 4 for x in hin)
    rec = {
        "value": weak_scaling_value(n_tasks / 2, steps, world, graph_ms),
        "unit": UNIT, "steps": steps, "ms_per_step": graph_ms / steps,
        "config": dict(mix_config(mx, world), lanes=lanes, plans_autotuned=bool(args.tune_plans),
                       windows=f"{n_separable} of {len(plans)} operators as separable plans "
                               "(pce_plan_create_separable: 2D node-grid hats), the rest dense",
                       step="all tasks (forward or adjoint each) as one CUDA-graph launch"),
        "roofline": {"kernel": "whole batch", "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak, "peak_source": ctx.peak_source(sm_max),
                     "traffic": None},
        "path_hbm": {"algorithmic_bytes_per_step": nbytes, "gbs": nbytes / step_s / 1e9,
                     "peak_gbs": ctx.hbm_peak, "peak_source": ctx.hbm_src,
                     "frac": nbytes / step_s / 1e9 / ctx.hbm_peak},
        "eager_lanes": {"value": weak_scaling_value(n_tasks / 2, esteps, world, eager_ms),
                        "ms_per_step": eager_ms / esteps},
        "comparator": ({"impl": "the same tasks issued one by one (pce_apply / pce_apply_adjoint) "
                                "on one stream, no lanes, no graph",
                        "value": weak_scaling_value(n_tasks / 2, qsteps, world, seq_ms),
                        "unit": UNIT, "ms_per_step": seq_ms / qsteps,
                        "speedup": (seq_ms / qsteps) / (graph_ms / steps)} if seq_ms else None),
        "e2e": {"value": weak_scaling_value(n_tasks / 2, e2e_steps, world, e2e_ms), "unit": UNIT,
                "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
                "how": "pinned host inputs -> device, graph, every output -> pinned host, every step; "
                       "two buffer sets on copy-in / compute / copy-out streams",
                "results_match_device_run": e2e_ok},
        "gpu_launches": launches * steps,
        "clocks": clocks,
        "wall_s": wall,
        "scratch_bytes": scratch,
        "model_makespan_ms": makespan,
        "tuning": tuned or None,
        "batch_tuning": batch_tuning,
        "accuracy": acc,
    }
    if args.cpu_baseline:
        rec["cpu_baseline"] = {k: v for k, v in oracle_mix_rate(mx, args.ref_seconds).items() if k != "seconds"}
    return rec


def top_line(args, rec: dict, world: int, config: dict) -> dict:
    """The contract's JSON line around a measurement record."""
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": rec["steps"],
            "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config}
    for k, v in rec.items():
        if k not in line and k not in ("config",):
            line[k] = v
    return line


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(synth.WORKLOADS) + [BATCH_WORKLOAD])
    ap.add_argument("--headline-only", action="store_true",
                    help="measure only the chosen workload (no sub-configs)")
    ap.add_argument("--configs", default=None,
                    help="comma-separated names of the sub-configs to measure (default: all)")
    ap.add_argument("--lanes", type=int, default=16, help="streams of the uneven batch")
    ap.add_argument("--autotune", dest="autotune", action="store_true", default=True,
                    help="autotune the plan(s) before timing (default)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--col-variant", type=int, default=None,
                    help="force the column variant of the plan (0, 1, 2) instead of autotuning")
    ap.add_argument("--row-variant", type=int, default=None, help="with --col-variant: the row variant")
    ap.add_argument("--backward", action="store_true", help="also time pce_backward (gradients)")
    ap.add_argument("--plan", default="auto", choices=["auto", "sectioned"],
                    help="plan: auto (separable for node-grid hats, else dense) or sectioned")
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
    if args.impl == "reference":
        reference_arm(args, args.workload, rank, world)
        return
    ctx = Ctx(rank, world)
    oracle_cache: dict = {}
    if args.workload == BATCH_WORKLOAD:
        rec = batch_arm(args, ctx)
        config = rec["config"] if rec else None
    else:
        pr = synth.workload(args.workload)
        rec = gpu_arm(args, pr, ctx, oracle_cache, headline=True)
        config = headline_config(pr, world)
        del pr
    line = top_line(args, rec, world, config) if rec else None
    if not args.headline_only and args.workload == HEADLINE:
        wanted = set(args.configs.split(",")) if args.configs else None
        subs = {}
        for name, wl, over in SUB_CONFIGS:
            if wanted is not None and name not in wanted:
                continue
            sargs = copy.copy(args)
            for k, v in over.items():
                setattr(sargs, k, v)
            if wl == BATCH_WORKLOAD:
                srec = batch_arm(sargs, ctx)
            else:
                spr = synth.workload(wl)
                srec = gpu_arm(sargs, spr, ctx, oracle_cache, headline=False)
                if srec is not None:
                    srec["config"] = headline_config(spr, world)
                del spr
            if srec is not None:
                subs[name] = srec
        if line is not None:
            line["configs"] = subs
    if line is not None:
        print(json.dumps(line), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
