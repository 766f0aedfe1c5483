"""Benchmark: polarization step time on the 96,000-atom water box (32,000 rigid waters,
98.7 A cube, PME grid 100^3, order 5, cutoff 7 A + 2 A list buffer, mixed precision, PCG
to 1e-5 D RMS).

One step = one pass of the whole hot path on a new configuration: neighbour blocks (rebuilt
every REBUILD steps, amortised), permanent field (real + PME + self), the guess, the PCG
solve, and the polarization energy and forces. The configurations are consecutive 2 fs
steps of a real trajectory, made in the untimed set-up by the library's rigid-water
integrator (--trajectory walk: the synthetic random walk instead). The reported value uses
the learned guess plus the adaptive (least-squares) extrapolation of its error over the
previous steps; the network is trained in the untimed set-up on ~2.3e6 solver-generated
pairs from water boxes of eight other seeds (the timed box is held out). The same steps
with the learned guess alone, the plain guess alpha E, the classical hold and the
classical adaptive predictor (alpha E in place of the network), other guesses, the
Jacobi/DIIS solver and the fixed-point mode are timed alongside. Inputs (every step's
positions) are resident on the device before timing; the L2 is flushed between timed
steps (the working set, ~60 MB, fits the 129 MB L2). `--impl reference` times the FP64
oracle on the host cores, full steps of the same workload. Other workloads:
`--workload chain23k | water1m | two_sets | replicas64 | precision | kernels`.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import contextlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "polarization solve ms/MD-step and PCG iters at 1e-5 D RMS, learned vs plain"
N_MOL, BOX, GRID, SEED, TRAJ_SEED, TRAIN_SEED = 32000, 98.7, (100, 100, 100), 1002, 2002, 3002
TRAIN_CONFIGS, TRAIN_STEPS, TRAIN_BATCH = 11, 1500, 16384    # ~1.06e6 (feature, dipole) pairs
CUTOFF, BUFFER, BETA, TOL = 7.0, 2.0, 0.5446, 1e-5
REBUILD = 20                       # steps between neighbour-list rebuilds
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
# FP32 operations per in-cutoff pair of the real-space matvec kernel (counted from its
# source: vector 6, r^2 5, rsqrt/r/r^-2 3, screening with erfc/exp 32, B1/B2 and U1/U2 10,
# Thole 8, R1/R2 4, two field updates 36; FMA = 2)
FLOPS_PER_PAIR_MATVEC = 104
# algorithmic FP32 work per in-range pair of the other pair kernels, counted from their source
# (FMA = 2, MUFU = 1; the radial terms once per pair): permanent field with quadrupoles (radial
# terms to R_3, both fields) and the real-space forces (radial terms to R_4, both multipole
# gradients, the dipole-dipole term, dU/dd and dU/dQ of both atoms)
FLOPS_PER_PAIR_FIELD = 174
FLOPS_PER_PAIR_FORCES = 467
MLP_FLOPS_PER_ATOM = 2 * (16 * 128 + 128 * 128 + 128 * 3)
# bytes per slot of one PCG iteration's vector kernels in the mixed mode (FP32 vectors as one
# float4 per slot, the diagonal and alpha as a float2): direction (r, diagonal/alpha, p in/out),
# q = A p (p, diagonal/alpha, FP64 real-space and FP32 reciprocal fields, q out, accumulator
# clear), update (p, q, diagonal/alpha, mu and r in/out)
PCG_VECTOR_BYTES_PER_SLOT = 56 + 100 + 104
WORKLOAD = "water_96000_atoms_98.7A_grid100_rc7+2_mixed_pcg1e-5"
HEADLINE_GUESS = "learned+adaptive"
GUESS_TEXT = {
    "learned+previous": "learned (16-128-128-3 BF16 MLP) plus its previous error: learned(t) + (mu - learned)(t-1) "
                        "(zero-order hold of the error, ap_extrapolate_guess)",
    "learned+adaptive": "learned(t) + e1 + c (e1 - e2), e = mu - learned at t-1, t-2, c the least-squares "
                        "coefficient of the three previous steps (ap_adaptive_guess)",
    "learned+extrapolated": "learned(t) + 2 (mu - learned)(t-1) - (mu - learned)(t-2)",
}
# kernels of this library one guess launches: the learned guess (alpha E, short-range field,
# features, MLP, assemble) plus the predictor of its error
GUESS_LAUNCHES = {"learned+previous": 6, "learned+adaptive": 7, "learned+extrapolated": 6, "direct+previous": 2,
                  "direct+adaptive": 3}
DIIS_DEPTH = 6          # window of the Jacobi/DIIS solver timed beside the PCG


def max_over_ranks(values, device=None):
    """Element-wise maximum over all ranks of a torch.distributed job (the slowest rank's
    time sets a weak-scaling step); the values themselves without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def captured_traffic():
    """DRAM bytes per launch of the real-space matvec from the committed ncu capture, if the
    kernel's sources are unchanged since (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "real_matvec_water96k.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    h = hashlib.sha256()
    for f in d["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return d["dram_bytes_per_launch"] if h.hexdigest()[:16] == d["source_sha256_16"] else None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _measured_field(key):
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh).get(key)
    return None


def _bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured burst"
    return 1900.0, "fallback"


def pcg_iteration_us(ctx, reps):
    """Time of one PCG iteration inside the solve graph: solves of exactly 4 and 12 iterations
    (an unreachable tolerance), each one graph launch timed with CUDA events, best of `reps`;
    (t12 - t4) / 8 in microseconds. Leaves the context's dipoles at a 12-iteration solve."""
    import torch
    stream = ctx.stream
    best = {}
    for k in (4, 12):
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.solve(tol=1e-30, max_iter=k, want_info=False)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        best[k] = min(ts)
    return (best[12] - best[4]) / 8 * 1e3


def kernel_rooflines(kern, per_launch_counts, n, n_pad, npairs, grid, fp32_peak=None):
    """Each timed kernel against its bound: FP32 ALU (pair kernels), HBM (spread, gather,
    convolution, PCG vectors; algorithmic bytes) or BF16 tensor (MLP)."""
    hbm, hbm_kind = _peaks()
    bf16, bf16_kind = _bf16_peak()
    k3 = grid[0] * grid[1] * grid[2]
    kc = grid[1] * grid[2] * (grid[0] // 2 + 1)
    work = {
        "real_matvec": ("alu", npairs * FLOPS_PER_PAIR_MATVEC),
        "real_field": ("alu", npairs * FLOPS_PER_PAIR_FIELD),
        "pair_forces": ("alu", npairs * FLOPS_PER_PAIR_FORCES),
        "spread_dipoles": ("hbm", n * 32 + k3 * 4),
        "gather_field": ("hbm", k3 * 4 + n * 28),
        "convolve": ("hbm", 2 * kc * 8 + kc * 4),
        "spread_multipoles": ("hbm", n * 64 + k3 * 4),
        "pcg_vectors": ("hbm", n_pad * PCG_VECTOR_BYTES_PER_SLOT),
        "mlp_forward": ("tensor", n * MLP_FLOPS_PER_ATOM),
    }
    out = {}
    for name, (bound, w) in work.items():
        if name not in kern:
            continue
        sec = kern[name] * 1e-3
        if bound == "hbm":
            ach, peak, unit, kind = w / sec / 1e9, hbm, "GB/s", hbm_kind
        elif bound == "alu":
            ach, unit = w / sec / 1e12, "TFLOP/s"
            peak, kind = (fp32_peak, "measured (ap_fp32_peak)") if fp32_peak else (FP32_PEAK_TFLOPS, "derived")
        else:
            ach, peak, unit, kind = w / sec / 1e12, bf16, "TFLOP/s", bf16_kind
        out[name] = {"bound": bound, "launch_us": round(kern[name] * 1e3, 2),
                     "launches_per_step": per_launch_counts.get(name, 1), "work_per_launch": int(w),
                     "achieved": round(ach, 3), "peak": round(peak, 2), "unit": unit, "peak_kind": kind,
                     "frac": round(ach / peak, 4)}
    return out


class Clocks:
    """nvidia-smi sampling during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            if os.path.exists(self.path):
                os.unlink(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_system():
    from paper_2011_01207_gb300 import synth
    return synth.water_box(N_MOL, BOX, SEED)


def trajectory(s, steps, seed=TRAJ_SEED, sigma_t=0.005, sigma_r=0.01):
    from paper_2011_01207_gb300 import synth
    out = [s.xyz.copy()]
    cur = s
    for k in range(1, steps):
        cur = synth.perturb(cur, seed + k, sigma_t, sigma_r)
        out.append(cur.xyz.copy())
    return np.stack(out)


MD_DT, MD_EQUIL, MD_T = 2.0, 300, 300.0    # fs, equilibration steps, K


def md_trajectory(s, steps, dev, grid, seed=TRAJ_SEED):
    """Positions of `steps` consecutive 2 fs steps of a real trajectory of the water box s: the
    library's rigid-water velocity Verlet (SHAKE/RATTLE) under its polarization forces and an
    O-O Lennard-Jones term, started from seeded 300 K velocities and equilibrated for
    MD_EQUIL steps with a weak Berendsen coupling (tau 50 fs, then 200 fs while recording)."""
    from paper_2011_01207_gb300 import binding, dynamics, synth
    c = binding.Context(s, cutoff=CUTOFF, buffer=BUFFER, beta=BETA, grid=grid, precision=binding.AP_MIXED,
                        device=dev)
    dyn = dynamics.RigidWaterMD(c, s, dt=MD_DT, rebuild_every=10, tol=TOL)
    dyn.start(synth.water_velocities(s, MD_T, seed))
    for _ in range(MD_EQUIL):
        dyn.step(target_temperature=MD_T, tau_fs=50.0)
    out = [c.xyz.cpu().numpy().copy()]
    for _ in range(1, steps):
        dyn.step(target_temperature=MD_T, tau_fs=200.0)
        out.append(c.xyz.cpu().numpy().copy())
    dyn.check()
    info = {"dt_fs": MD_DT, "equilibration_steps": MD_EQUIL, "temperature_K": round(dyn.temperature(), 1)}
    c.close()
    return np.stack(out), info


def pairs_within(xyz, box, rc):
    from scipy.spatial import cKDTree
    w = np.mod(xyz, box)
    w[w >= box] = 0.0
    return len(cKDTree(w, boxsize=box).query_pairs(rc, output_type="ndarray"))


def launches_per_step(iters, n, rebuild_frac, guess_launches):
    """Kernels of this library launched by one step (cuFFT's own kernels not counted)."""
    pad = 1 if n % 32 else 0
    field = 8 + pad + 5                   # load, filter, work offsets, work fill, pair masks, 3 prefix
    #                                       scans, [pad]; spread, convolve, gather, pair field, assemble
    guess = guess_launches
    solve = 1 + 4 + 1 + 1 + 7 * iters + 1  # guess, matvec(4), residual (+ state), cond, 7/iter, unsort
    forces = 10
    build = 14 * rebuild_frac
    return field + guess + solve + forces + build


# step workloads: the timed system, its PME grid, and the systems the learned guess is trained
# on (other seeds: the timed box is held out). The 1,065,000-atom box uses the network trained
# on 96,000-atom boxes (the features are local, so it transfers).
STEP_WORKLOADS = {
    "water96k": {"name": WORKLOAD, "system": ("water", N_MOL, BOX, SEED), "grid": GRID,
                 "train": [("water", N_MOL, BOX, 1002 + 100 * k) for k in range(1, 9)], "train_grid": GRID,
                 "per_box": 3, "all_guesses": True},
    "chain23k": {"name": "chain_23558_atoms_62.2A_grid64_rc7+2_mixed_pcg1e-5",
                 "system": ("chain", 2489, 7023, 62.2, 1003), "grid": (64, 64, 64),
                 "train": [("chain", 2489, 7023, 62.2, sd) for sd in (1113, 1123, 1133, 1143, 1153, 1163)],
                 "train_grid": (64, 64, 64), "per_box": 8, "all_guesses": False},
    "water1m": {"name": "water_1065000_atoms_221.6A_grid224_rc7+2_mixed_pcg1e-5",
                "system": ("water", 355000, 221.6, 1004), "grid": (224, 224, 224),
                "train": [("water", N_MOL, BOX, 1002 + 100 * k) for k in range(1, 9)], "train_grid": GRID,
                "per_box": 3, "all_guesses": False},
}


def make_system_spec(spec):
    from paper_2011_01207_gb300 import synth
    if spec[0] == "water":
        return synth.water_box(spec[1], spec[2], spec[3])
    return synth.solvated_chain(spec[1], spec[2], spec[3], spec[4])


def train_learned_guess(wl, dev):
    """Solver-generated (feature, dipole) pairs from the workload's training systems (other
    seeds than the timed one; configurations from large random moves, lists rebuilt at
    each), then Adam on the GPU kernels. Returns (trainer, losses, pairs, seconds)."""
    import torch
    from paper_2011_01207_gb300 import binding, learned
    t0 = time.perf_counter()
    feats, tgts = [], []
    for k, spec in enumerate(wl["train"]):
        ts = make_system_spec(spec)
        confs = trajectory(ts, wl["per_box"], seed=TRAIN_SEED + 100 * k, sigma_t=0.05, sigma_r=0.1)
        c = binding.Context(ts, cutoff=CUTOFF, buffer=BUFFER, beta=BETA, grid=wl["train_grid"],
                            precision=binding.AP_MIXED, device=dev)
        for xyz in confs:
            c.set_positions(xyz)
            c.build()
            f, t = learned.collect(c, [xyz], tol=1e-8)
            feats.append(f)
            tgts.append(t)
        c.close()
    feat, tgt = torch.cat(feats), torch.cat(tgts)
    trainer = learned.Trainer(seed=7, device=dev)
    losses = trainer.fit(feat, tgt, steps=TRAIN_STEPS, batch=TRAIN_BATCH, lr=3e-3, lr_final=3e-4)
    return trainer, losses, int(feat.shape[0]), time.perf_counter() - t0


def fp32_peak_derived(sm_count, sm_max_mhz):
    """FP32 FMA peak from unit counts and clock: SMs x 128 FP32 lanes x 2 flops x max SM clock."""
    return sm_count * 128 * 2 * sm_max_mhz * 1e6 / 1e12


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2011_01207_gb300 import binding, build as _build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    _build.build_library()
    dev = torch.device("cuda", local)
    wl = STEP_WORKLOADS[args.workload]
    grid = wl["grid"]
    s = make_system_spec(wl["system"])
    total = args.warmup + args.steps
    use_md = args.trajectory == "md" and wl["system"][0] == "water"
    if use_md:
        traj, traj_info = md_trajectory(s, total, dev, grid)
        s = s.copy()
        s.xyz = traj[0].copy()
    else:
        traj, traj_info = trajectory(s, total), {"kind": "random walk"}
    pos = torch.tensor(traj, device=dev)                       # [steps, N, 3], resident before timing
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    # learned guess: trained in the untimed set-up on boxes of other seeds (held-out timed box)
    trainer, tr_loss, n_train, t_train = train_learned_guess(wl, dev)
    ctx = binding.Context(s, cutoff=CUTOFF, buffer=BUFFER, beta=BETA, grid=grid, precision=binding.AP_MIXED,
                          device=dev)
    ctx.build()
    tuned = None
    if not args.no_autotune:
        ctx.permanent_field(out=False)
        tuned = binding.ap_autotune(ctx.ctx, 3)   # launch shapes, untimed set-up
    mu0 = torch.zeros((s.n, 3), dtype=torch.float64, device=dev)

    # ring buffers for the trajectory guesses: converged dipoles and base guesses of the
    # current and the last three steps (written in place by the library, no copies)
    RING = 4
    ring_mu = [torch.zeros((s.n, 3), dtype=torch.float64, device=dev) for _ in range(RING)]
    ring_g = [torch.zeros((s.n, 3), dtype=torch.float64, device=dev) for _ in range(RING)]
    scratch = torch.zeros(binding.AP_ADAPTIVE_SCRATCH, dtype=torch.float64, device=dev)
    hist = {"count": 0}

    def step(k, xyz, use_learned, ctx=ctx, solver="pcg"):
        """use_learned: True (MLP), False (alpha E), "zero", "extrapolated" (2 mu(t-1) -
        mu(t-2)), "direct+previous" (alpha E plus its previous error, the classical hold:
        alpha E(t) + (mu - alpha E)(t-1)), "direct+adaptive" (alpha E plus the adaptive
        extrapolation of its error, the classical counterpart of the headline),
        "learned+extrapolated" (the learned guess plus the
        linear extrapolation of its error over the two previous steps), "learned+previous"
        (plus its previous error) or "learned+adaptive" (plus its error extrapolated with the
        least-squares coefficient of the three previous steps, ap_adaptive_guess; the previous
        error while fewer steps exist); the trajectory guesses fall back to their base guess
        until enough previous steps exist."""
        if k % REBUILD == 0:
            binding.build_neighbour_blocks(ctx.ctx, xyz, ctx.excl_off, ctx.excl_atoms, ctx.n_excl)
        binding.permanent_field(ctx.ctx, xyz, ctx.mpole, ctx.frame, ctx.alpha, None)
        guess, out = None, ctx.mu
        ready = hist["count"] >= 2
        if use_learned is True:
            binding.ap_learned_guess(ctx.ctx, trainer.packed, mu0)
            guess = mu0
        elif use_learned == "zero":
            mu0.zero_()
            guess = mu0
        elif use_learned == "extrapolated":
            out = ring_mu[k % RING]
            if ready:
                binding.ap_extrapolate_guess(mu0, ring_mu[(k - 1) % RING], ring_mu[(k - 2) % RING])
                guess = mu0
        elif use_learned == "learned+extrapolated":
            out = ring_mu[k % RING]
            binding.ap_learned_guess(ctx.ctx, trainer.packed, ring_g[k % RING])
            guess = ring_g[k % RING]
            if ready:
                binding.ap_extrapolate_guess(mu0, ring_mu[(k - 1) % RING], ring_mu[(k - 2) % RING], base=ring_g[k % RING],
                                             base1=ring_g[(k - 1) % RING], base2=ring_g[(k - 2) % RING])
                guess = mu0
        elif use_learned in ("learned+adaptive", "direct+adaptive"):
            out = ring_mu[k % RING]
            g = ring_g[k % RING]
            if use_learned == "learned+adaptive":
                binding.ap_learned_guess(ctx.ctx, trainer.packed, g)
            else:
                binding.ap_direct_guess(ctx.ctx, g)
            guess = g
            m1, m2, m3 = (ring_mu[(k - j) % RING] for j in (1, 2, 3))
            g1, g2, g3 = (ring_g[(k - j) % RING] for j in (1, 2, 3))
            if hist["count"] >= 3:
                binding.ap_adaptive_guess(mu0, m1, m2, m3, scratch, base=g, base1=g1, base2=g2, base3=g3)
                guess = mu0
            elif hist["count"] >= 1:
                binding.ap_extrapolate_guess(mu0, m1, m1, base=g, base1=g1, base2=g1)
                guess = mu0
        elif use_learned in ("learned+previous", "direct+previous"):
            # zero-order hold of the base guess's error: g(t) + (mu - g)(t-1), with g the
            # learned guess or (the classical control) alpha E
            out = ring_mu[k % RING]
            if use_learned == "learned+previous":
                binding.ap_learned_guess(ctx.ctx, trainer.packed, ring_g[k % RING])
            else:
                binding.ap_direct_guess(ctx.ctx, ring_g[k % RING])
            guess = ring_g[k % RING]
            if hist["count"] >= 1:
                binding.ap_extrapolate_guess(mu0, ring_mu[(k - 1) % RING], ring_mu[(k - 1) % RING], base=ring_g[k % RING],
                                             base1=ring_g[(k - 1) % RING], base2=ring_g[(k - 1) % RING])
                guess = mu0
        if solver == "diis":
            binding.induced_dipoles_diis(ctx.ctx, guess, TOL, 200, DIIS_DEPTH, out, want_info=False)
        else:
            binding.induced_dipoles_pcg(ctx.ctx, guess, TOL, 200, out, want_info=False)
        binding.polarization_energy_forces(ctx.ctx, out, ctx.energy, ctx.forces)
        hist["count"] += 1

    eps0 = {}       # initial residual (Debye) of every timed step, per guess

    def timed(use_learned, tag, c=ctx, solver="pcg", positions=None):
        pos_ = pos if positions is None else positions
        hist["count"] = 0
        it_, ts = [], []
        for k in range(args.warmup):
            step(k, pos_[k], use_learned, c, solver)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.nvtx.range_push(tag)
        for k in range(args.warmup, total):
            flush.fill_(k & 0xff)                                    # untimed: evict the L2
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(k, pos_[k], use_learned, c, solver)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
            inf = binding.ap_solve_info_last(c.ctx)
            it_.append(inf.iterations)
            eps0[tag] = eps0.get(tag, []) + [inf.eps_initial]
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        return ts, it_

    clocks = Clocks(local)
    clocks.start()
    # headline: the learned guess plus its error at the previous step
    t_wall = time.perf_counter()
    times, iters = timed(HEADLINE_GUESS, "timed_steps")
    t_wall = time.perf_counter() - t_wall
    times_learned, iters_learned = timed(True, "timed_steps_learned_only")
    times_plain, iters_plain = timed(False, "timed_steps_plain")
    times_hold, iters_hold = timed("direct+previous", "timed_steps_classical_hold")
    times_cad, iters_cad = timed("direct+adaptive", "timed_steps_classical_adaptive")
    others = {}
    if wl["all_guesses"]:
        others["learned+previous"] = timed("learned+previous", "timed_steps_learned_previous")
        others["zero"] = timed("zero", "timed_steps_zero")
        others["extrapolated"] = timed("extrapolated", "timed_steps_extrapolated")

        others["learned+extrapolated"] = timed("learned+extrapolated", "timed_steps_learned_extrapolated")
        # the same steps with the Jacobi/DIIS solver in place of the PCG
        others["diis"] = timed(HEADLINE_GUESS, "timed_steps_diis", solver="diis")
        # the same steps in the fixed-point accumulation mode (AP_FIXED)
        ctx_fx = binding.Context(s, cutoff=CUTOFF, buffer=BUFFER, beta=BETA, grid=grid, precision=binding.AP_FIXED,
                                 device=dev)
        others["fixed"] = timed(HEADLINE_GUESS, "timed_steps_fixed", ctx_fx)
        kern_fx = {k: round(binding.ap_time_kernel(ctx_fx.ctx, k, 20), 4) for k in
                   ("real_matvec", "spread_dipoles", "real_field", "pair_forces", "spread_multipoles")}
        ctx_fx.close()
    walk = {}
    if use_md:
        # the same two guesses along the synthetic random walk of the same box (the workload of
        # earlier measurements), for comparison
        pos_walk = torch.tensor(trajectory(s, total), device=dev)
        ctx.xyz.copy_(pos_walk[0])
        ctx.build()
        tw, iw = timed(HEADLINE_GUESS, "timed_steps_walk", positions=pos_walk)
        twp, iwp = timed(False, "timed_steps_walk_plain", positions=pos_walk)
        walk = {"walk_ms_per_step": round(float(np.mean(tw)), 4), "walk_pcg_iters": float(np.mean(iw)),
                "walk_plain_ms_per_step": round(float(np.mean(twp)), 4), "walk_plain_pcg_iters": float(np.mean(iwp))}
        del pos_walk
        ctx.xyz.copy_(pos[0])
        ctx.build()
    clk = clocks.stop()
    ms = float(np.mean(times))
    ms_plain = float(np.mean(times_plain))
    ms_learned = float(np.mean(times_learned))
    ms_hold = float(np.mean(times_hold))
    ms_cad = float(np.mean(times_cad))
    ms, ms_plain, ms_learned, ms_hold, ms_cad = max_over_ranks([ms, ms_plain, ms_learned, ms_hold, ms_cad], dev)

    # end to end through the public API with host buffers: every step's positions copied in
    # from pinned host memory, forces and energy copied out, inside the timed region; the
    # same trajectory and guess as the headline
    host_traj = torch.tensor(traj, dtype=torch.float64).pin_memory()
    host_f = torch.empty((s.n, 3), dtype=torch.float64).pin_memory()
    host_e = torch.empty(1, dtype=torch.float64).pin_memory()
    dev_pos = torch.empty((s.n, 3), dtype=torch.float64, device=dev)
    e2e = []
    hist["count"] = 0
    for k in range(total):
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dev_pos.copy_(host_traj[k], non_blocking=True)
        step(k, dev_pos, HEADLINE_GUESS)
        host_f.copy_(ctx.forces, non_blocking=True)
        host_e.copy_(ctx.energy, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if k >= args.warmup:
            e2e.append(a.elapsed_time(b))
    e2e_ms = max_over_ranks([float(np.mean(e2e))], dev)[0]

    # every kernel: per-launch durations with CUDA events on the launch stream
    it_mean = float(np.mean(iters))
    kern = {k: binding.ap_time_kernel(ctx.ctx, k, 30) for k in
            ("real_matvec", "spread_dipoles", "gather_field", "convolve", "real_field", "spread_multipoles",
             "pair_forces")}
    kern["pcg_vectors"] = binding.ap_time_kernel(ctx.ctx, "pcg_vectors", 30)
    # one application of T as inside the solve (both branches), its reciprocal branch alone
    # and that branch's transforms: what bounds an iteration beside the vector kernels
    operator_us = {k: round(binding.ap_time_kernel(ctx.ctx, k, 30) * 1e3, 2)
                   for k in ("dipole_operator", "pme_dipoles", "fft_roundtrip", "real_matvec")}
    operator_us["pcg_vectors"] = round(kern["pcg_vectors"] * 1e3, 2)
    operator_us["pcg_iteration"] = round(pcg_iteration_us(ctx, 10), 2)
    feat_t = torch.randn((s.n, 16), dtype=torch.float32, device=dev)
    y_t = torch.empty((s.n, 3), dtype=torch.float32, device=dev)
    binding.ap_mlp_forward(trainer.packed, feat_t, y_t)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(30):
        binding.ap_mlp_forward(trainer.packed, feat_t, y_t)
    ev1.record(stream)
    ev1.synchronize()
    kern["mlp_forward"] = ev0.elapsed_time(ev1) / 30
    per_step = {"real_matvec": kern["real_matvec"] * (it_mean + 1),
                "spread_dipoles": kern["spread_dipoles"] * (it_mean + 1),
                "gather_field": kern["gather_field"] * (it_mean + 1),
                "real_field": kern["real_field"], "spread_multipoles": kern["spread_multipoles"],
                "pair_forces": kern["pair_forces"]}
    npairs = pairs_within(traj[-1], s.box, CUTOFF)
    hbm_peak, peak_kind = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = clk.get("sm_max_mhz") or _measured_field("sm_max_mhz") or 2070.0
    fp32_derived = fp32_peak_derived(sm_count, sm_max)
    fp32_fma, _ = binding.ap_fp32_peak(10)
    flop = npairs * FLOPS_PER_PAIR_MATVEC
    achieved = flop / (kern["real_matvec"] * 1e-3) / 1e12
    roofline = {"kernel": "real_matvec (a5 real-space pair kernel)", "bound": "alu", "achieved": round(achieved, 3),
                "peak": round(fp32_derived, 2), "unit": "TFLOP/s", "frac": round(achieved / fp32_derived, 4),
                "traffic": captured_traffic() if args.workload == "water96k" else None,
                "traffic_unit": "bytes per launch (ncu, cold caches)", "flop_per_launch": flop,
                "pairs_in_cutoff": npairs, "launch_ms": round(kern["real_matvec"], 4),
                "peak_note": f"FP32 FMA peak derived from unit counts and clock: {sm_count} SMs (queried) x 128 "
                             f"lanes x 2 x {sm_max:.0f} MHz (max SM clock)",
                "sm_count": sm_count, "peak_measured_fma": round(fp32_fma, 2),
                "frac_of_measured_fma": round(achieved / fp32_fma, 4),
                "hbm_peak_gbs": hbm_peak, "hbm_peak_kind": peak_kind}
    counts = {"real_matvec": it_mean + 1, "spread_dipoles": it_mean + 2, "gather_field": it_mean + 1,
              "convolve": it_mean + 3, "pcg_vectors": it_mean}
    kernels = kernel_rooflines(kern, counts, s.n, (s.n + 31) // 32 * 32, npairs, grid, fp32_peak=fp32_derived)
    nb, nt, ne = ctx.stats()
    cmp = {"plain_ms_per_step": round(ms_plain, 4), "plain_pcg_iters": float(np.mean(iters_plain)),
           "learned_only_ms_per_step": round(ms_learned, 4), "learned_only_pcg_iters": float(np.mean(iters_learned)),
           "classical_hold_ms_per_step": round(ms_hold, 4), "classical_hold_pcg_iters": float(np.mean(iters_hold)),
           "classical_adaptive_ms_per_step": round(ms_cad, 4),
           "classical_adaptive_pcg_iters": float(np.mean(iters_cad)),
           "headline_pcg_iters": it_mean,
           # the initial residual of each guess (Debye RMS of alpha r0): the guess quality itself,
           # which the whole-number iteration counts show only in steps
           "headline_eps0_debye": float(f"{np.mean(eps0['timed_steps']):.4e}"),
           "plain_eps0_debye": float(f"{np.mean(eps0['timed_steps_plain']):.4e}"),
           "learned_only_eps0_debye": float(f"{np.mean(eps0['timed_steps_learned_only']):.4e}"),
           "classical_hold_eps0_debye": float(f"{np.mean(eps0['timed_steps_classical_hold']):.4e}"),
           "classical_adaptive_eps0_debye": float(f"{np.mean(eps0['timed_steps_classical_adaptive']):.4e}")}
    config = {"workload": wl["name"], "atoms": s.n, "guess": GUESS_TEXT[HEADLINE_GUESS],
              "pcg_iters_mean": it_mean, "pcg_iters": [int(min(iters)), int(max(iters))], **cmp,
              "classical_hold_guess": "alpha E(t) + (mu - alpha E)(t-1) (ap_direct_guess + ap_extrapolate_guess)",
              "classical_adaptive_guess": "alpha E(t) + the adaptive extrapolation of (mu - alpha E) over the three "
                                          "previous steps (ap_direct_guess + ap_adaptive_guess): the headline's "
                                          "predictor without the network",
              **walk, "learned_train_boxes": len(wl["train"]), "learned_train_pairs": n_train,
              "learned_held_out": "the timed box's seed is not among the training boxes' seeds",
              "trajectory": ("rigid-water MD, 2 fs steps (ap_md_kick_drift / ap_md_kick, polarization + O-O "
                             "Lennard-Jones forces, Berendsen 300 K)") if use_md else
                            "random walk (rigid moves ~N(0, 0.005 A), ~N(0, 0.01 rad) per step)",
              "trajectory_temperature_K": traj_info.get("temperature_K"),
              "rebuild_every": REBUILD, "l2": "flushed between timed steps (256 MB write)", "blocks": nb, "tiles": nt,
              "launch_shapes": ({"matvec_ctas_per_sm": tuned[0], "pme_threads": tuned[1], "by": "ap_autotune"}
                                if tuned else {"matvec_ctas_per_sm": 0, "pme_threads": 128, "by": "defaults"}),
              "excl_tiles": ne, "replicas": world, "parallelism": "replicas" if world > 1 else "1 GPU",
              "learned_training": {"pairs": n_train, "adam_steps": TRAIN_STEPS, "batch": TRAIN_BATCH,
                                   "loss_first": round(float(tr_loss[0]), 5),
                                   "loss_last": round(float(np.mean(tr_loss[-20:])), 5), "seconds": round(t_train, 2)}}
    if others:
        og = {}
        tags = {"zero": "timed_steps_zero", "extrapolated": "timed_steps_extrapolated",
                "learned+previous": "timed_steps_learned_previous",
                "learned+extrapolated": "timed_steps_learned_extrapolated"}
        for key, txt in (("zero", "zero"), ("extrapolated", "2 mu(t-1) - mu(t-2) from the previous steps' solves"),
                         ("learned+previous", GUESS_TEXT["learned+previous"]),
                         ("learned+extrapolated", GUESS_TEXT["learned+extrapolated"])):
            ts_, it_ = others[key]
            og[key] = {"ms_per_step": round(float(np.mean(ts_)), 4), "pcg_iters_mean": float(np.mean(it_)),
                       "eps0_debye": float(f"{np.mean(eps0[tags[key]]):.4e}"), "guess": txt}
        for key, name in (("extrapolated", "extrapolated"), ("learned+previous", "learned_previous")):
            config[f"{name}_ms_per_step"] = og[key]["ms_per_step"]
            config[f"{name}_pcg_iters"] = og[key]["pcg_iters_mean"]
        config["other_guesses"] = og
        ts_, it_ = others["diis"]
        config["other_solvers"] = {"jacobi_diis": {"ms_per_step": round(float(np.mean(ts_)), 4),
                                                   "updates_mean": float(np.mean(it_)), "depth": DIIS_DEPTH,
                                                   "t_applications_mean": float(np.mean(it_)) + 1,
                                                   "guess": "as the headline"},
                                   "pcg": {"t_applications_mean": it_mean + 1}}
        ts_, it_ = others["fixed"]
        config["fixed_point"] = {"ms_per_step": round(float(np.mean(ts_)), 4), "pcg_iters_mean": float(np.mean(it_)),
                                 "guess": "as the headline",
                                 "accumulation": "64-bit fixed point (AP_FIXED), bitwise reproducible",
                                 "kernel_ms": kern_fx}
    launches = GUESS_LAUNCHES[HEADLINE_GUESS]
    result = {
        "metric": METRIC, "value": round(ms, 4), "unit": "ms/step", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 pair/PME arithmetic, f64 accumulation", "data": "synthetic",
        "config": config, **cmp,
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms/step", "h2d_bytes_per_step": int(s.n * 3 * 8),
                "d2h_bytes_per_step": int(s.n * 3 * 8 + 8)},
        "gpu_launches": int(round(launches_per_step(it_mean, s.n, 1.0 / REBUILD, launches) * args.steps)),
        "kernel_ms": {k: round(v, 4) for k, v in kern.items()},
        "kernel_ms_per_step": {k: round(v, 4) for k, v in per_step.items()},
        "roofline": roofline,
        "kernels": kernels,
        "operator_us": operator_us,
        "clocks": clk,
        "wall_s_timed_region": round(t_wall, 3),
    }
    if rank == 0 and not args.no_cpu and args.workload == "water96k":
        # the library's outputs at the first configuration (plain guess, the benchmark's
        # tolerance), for its errors against the oracle there
        ctx.set_positions(traj[0])
        ctx.build()
        ctx.permanent_field()
        ctx.solve(tol=TOL, max_iter=200)
        e_g, f_g, v_g = ctx.energy_forces(virial=True)
        gpu_out = (ctx.field.cpu().numpy(), ctx.mu.cpu().numpy(), float(e_g.item()), f_g.cpu().numpy(),
                   v_g.cpu().numpy())
        ctx.close()
        base, errors = cpu_baseline(s, gpu_out)
        result["cpu_baseline"] = base
        if errors:
            config.update({k: float(f"{v:.3e}") for k, v in errors.items()})
    else:
        ctx.close()
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


def make_replicas(n_rep=64, lo=648, hi=24000, seed=1005):
    """Seeded replicas with sizes uniform in [lo, hi] atoms, alternating water boxes (even
    index) and solvated chains (odd index: a random-walk chain of a tenth of the atoms in
    water, at the 23,558-atom chain box's density); PME grid = the smallest even 7-smooth
    K >= L / 1 A."""
    from paper_2011_01207_gb300 import synth
    sizes = synth.replica_sizes(n_rep, lo, hi, seed)
    out = []
    for k, n in enumerate(sizes):
        if k % 2 == 0:
            nmol = int(n) // 3
            L = synth.water_cfg(nmol)
            s = synth.water_box(nmol, L, seed + 10 * k)
        else:
            nc = max(30, int(n) // 10)
            nw = (int(n) - nc) // 3
            L = ((nc + 3 * nw) / 0.0979) ** (1.0 / 3.0)
            s = synth.solvated_chain(nc, nw, L, seed + 10 * k)
        K = next(k2 for k2 in range(int(np.ceil(L)), 4 * int(np.ceil(L)) + 8) if k2 % 2 == 0 and _smooth7(k2))
        out.append((s, (K, K, K)))
    return out


def _smooth7(k):
    for p in (2, 3, 5, 7):
        while k % p == 0:
            k //= p
    return k == 1


def run_replicas(args):
    """64 independent replicas advanced together: one CUDA-graph launch per batch step."""
    import torch
    from paper_2011_01207_gb300 import binding, build as _build, learned, synth
    _build.build_library()
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    reps = make_replicas()
    t_gen = time.perf_counter() - t0
    total = args.warmup + args.steps
    ctxs, trajs = [], []
    for k, (s, grid) in enumerate(reps):
        c = binding.Context(s, cutoff=CUTOFF, buffer=BUFFER, beta=BETA, grid=grid, precision=binding.AP_MIXED,
                            device=dev, stream=torch.cuda.Stream(dev))
        ctxs.append(c)
        trajs.append(torch.tensor(trajectory(s, total, seed=TRAJ_SEED + 1000 * k), device=dev))
    # training pairs: one separate configuration per replica (~0.8e6 pairs), then tuning
    feats, tgts = [], []
    for k, ((s, grid), c) in enumerate(zip(reps, ctxs)):
        with torch.cuda.stream(c.stream):
            c.build()
            f, t = learned.collect(c, [synth.perturb(s, 77 + k, 0.05, 0.1).xyz], tol=1e-8)
            feats.append(f)
            tgts.append(t)
    torch.cuda.synchronize()
    feat, tgt = torch.cat(feats), torch.cat(tgts)
    trainer = learned.Trainer(seed=7, device=dev)
    trainer.fit(feat, tgt, steps=TRAIN_STEPS, batch=TRAIN_BATCH, lr=3e-3, lr_final=3e-4)
    del feat, tgt, feats, tgts
    tuned = []
    for c, tr in zip(ctxs, trajs):
        with torch.cuda.stream(c.stream):
            c.xyz.copy_(tr[0])
            c.build()
            c.permanent_field(out=False)
            binding.ap_learned_guess(c.ctx, trainer.packed, c.mu)   # sets MLP kernel attributes
            tuned.append(binding.ap_autotune(c.ctx, 3))
    torch.cuda.synchronize()
    batch = binding.Batch(ctxs)
    batch.capture(tol=TOL, max_iter=200, packed=trainer.packed)
    # learned plus the adaptive extrapolation of its error over the three previous batch steps
    # (history kept inside the graph)
    batch_h = binding.Batch(ctxs)
    batch_h.capture(tol=TOL, max_iter=200, packed=trainer.packed, history="adaptive")
    main = torch.cuda.Stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def set_step(k):
        for c, tr in zip(ctxs, trajs):
            c.xyz.copy_(tr[k])

    def one_by_one():
        # the same replica steps through the public calls, each replica on its own stream
        for c, mu0 in zip(ctxs, batch._keep):
            with torch.cuda.stream(c.stream):
                binding.permanent_field(c.ctx, c.xyz, c.mpole, c.frame, c.alpha, None)
                binding.ap_learned_guess(c.ctx, trainer.packed, mu0)
                binding.induced_dipoles_pcg(c.ctx, mu0, TOL, 200, c.mu, want_info=False)
                binding.polarization_energy_forces(c.ctx, c.mu, c.energy, c.forces)

    def timed(fn):
        out = []
        for k in range(total):
            set_step(k)
            flush.fill_(k & 0xff)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            fn()
            torch.cuda.synchronize()
            b.record(main)
            b.synchronize()
            if k >= args.warmup:
                out.append(a.elapsed_time(b))
        return float(np.mean(out))

    clocks = Clocks(0)
    clocks.start()
    ms_hist = timed(lambda: batch_h.launch(main))
    iters_hist = [binding.ap_solve_info_last(c.ctx).iterations for c in ctxs]
    ms_graph = timed(lambda: batch.launch(main))
    clk = clocks.stop()
    iters = [binding.ap_solve_info_last(c.ctx).iterations for c in ctxs]
    ms_seq = timed(one_by_one)
    atoms = int(sum(s.n for s, _ in reps))
    print(json.dumps({
        "metric": METRIC, "value": round(ms_hist, 4), "unit": "ms per batch step (64 replicas)", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_hist, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 pair/PME arithmetic, f64 accumulation",
        "data": "synthetic",
        "config": {"workload": "replicas_64_water_and_chain_sizes_648-24000_mixed_learned_pcg1e-5",
                   "replicas": len(reps), "atoms_total": atoms, "sizes": [int(s.n) for s, _ in reps],
                   "grids": [int(g[0]) for _, g in reps], "pcg_iters": iters_hist,
                   "guess": "learned plus the adaptive (least-squares) extrapolation of its error over the three previous batch steps",
                   "learned_only": {"ms_per_batch_step": round(ms_graph, 4), "pcg_iters": iters,
                                    "one_by_one_ms_per_batch_step": round(ms_seq, 4),
                                    "graph_speedup": round(ms_seq / ms_graph, 3)},
                   "autotuned_shapes": tuned, "generation_s": round(t_gen, 1),
                   "atom_steps_per_s": round(atoms / (ms_hist * 1e-3), 1),
                   "l2": "flushed between timed steps (256 MB write)"},
        "clocks": clk,
    }))
    batch.close()
    batch_h.close()
    for c in ctxs:
        c.close()


# ---- the oracle timed on the host cores ---------------------------------------------------
# A full oracle step (pairs, permanent field, PCG from alpha E to the tolerance, energy,
# forces) through the oracle's own code path, Oracle.permanent_field / pcg / energy / forces,
# unchanged. Only its pair sums and smooth-PME passes are spread over the host cores: every
# worker process owns a range of target atoms (their ordered pairs, found with a periodic k-d
# tree, and their scale factors from the oracle's pair module) and runs the oracle's real-space
# functions on it, or spreads / gathers the smooth-PME grid for those atoms with the oracle's
# spme functions; the parent sums the parts, transforms the grid and runs everything else.


def _oracle_worker(conn, lo, hi):
    """One worker of the host-core harness: commands from the parent over a pipe."""
    from scipy.spatial import cKDTree
    from oracle import pairs as opairs, realspace, spme
    st = {}
    while True:
        msg = conn.recv()
        cmd = msg[0]
        try:
            if cmd == "stop":
                conn.send(("ok", None))
                break
            if cmd == "setup":                      # system arrays and this worker's pairs
                xyz, box, rc, excl, n = msg[1:]
                w = np.mod(xyz, box)
                w[w >= box] = 0.0
                tree = cKDTree(w, boxsize=box)
                nb = tree.query_ball_point(w[lo:hi], rc)
                I = np.repeat(np.arange(lo, hi), [len(x) for x in nb])
                J = np.fromiter((j for x in nb for j in x), dtype=np.int64, count=len(I))
                keep = I != J
                I, J = I[keep], J[keep]
                R = xyz[I] - xyz[J]
                R -= box * np.round(R / box)
                keep = np.einsum("ij,ij->i", R, R) < rc * rc
                I, J, R = I[keep], J[keep], R[keep]
                st.update(xyz=xyz, box=box, n=n, I=I, J=J, R=R, sigma=opairs.scale_of_pairs(I, J, excl, n, R, box))
                conn.send(("ok", len(I)))
            elif cmd == "real_field":
                conn.send(("ok", realspace.real_field(st["n"], st["I"], st["J"], st["R"], st["sigma"], *msg[1:])))
            elif cmd == "real_dipole_field":
                conn.send(("ok", realspace.real_dipole_field(st["n"], st["I"], st["J"], st["R"], *msg[1:])))
            elif cmd == "real_forces":              # the last argument is the virial flag
                conn.send(("ok", realspace.real_forces(st["n"], st["I"], st["J"], st["R"], st["sigma"], *msg[1:-1],
                                                       virial=msg[-1])))
            elif cmd == "spread":                   # this worker's atoms only
                K, order, q, dip, quad = msg[1:]
                conn.send(("ok", spme.spread(st["xyz"][lo:hi], st["box"], K, order, q, dip, quad)))
            elif cmd == "gather":
                phi, K, order, max_order = msg[1:]
                conn.send(("ok", spme.gather(phi, st["xyz"][lo:hi], st["box"], K, order, max_order)))
            else:
                conn.send(("err", f"unknown command {cmd}"))
        except Exception as e:                      # reported to the parent, which raises
            conn.send(("err", repr(e)))


class HostOracle:
    """The oracle on `procs` host processes (spawn start method: safe after CUDA use)."""

    def __init__(self, procs):
        import multiprocessing as mp
        self.procs = procs
        self.ctx = mp.get_context("spawn")
        self.workers = []

    def start(self, n):
        bounds = np.linspace(0, n, self.procs + 1).astype(int)
        self.bounds = [(int(bounds[k]), int(bounds[k + 1])) for k in range(self.procs)]
        for k in range(self.procs):
            a, b = self.ctx.Pipe()
            pr = self.ctx.Process(target=_oracle_worker, args=(b, int(bounds[k]), int(bounds[k + 1])), daemon=True)
            pr.start()
            self.workers.append((pr, a))

    def call(self, *msg, sliced=()):
        """Send msg to every worker (the arguments at positions `sliced` cut to the worker's
        atoms) and collect the results in worker order."""
        for (_, c), (lo, hi) in zip(self.workers, self.bounds):
            c.send(tuple(m[lo:hi] if k in sliced else m for k, m in enumerate(msg)))
        out = []
        for _, c in self.workers:
            status, val = c.recv()
            if status != "ok":
                raise RuntimeError(f"oracle worker failed: {val}")
            out.append(val)
        return out

    def stop(self):
        for pr, c in self.workers:
            try:
                c.send(("stop",))
                c.recv()
            except Exception:
                pass
            pr.join(timeout=10)
        self.workers = []

    @contextlib.contextmanager
    def installed(self):
        """While active, the oracle model's pair enumeration, real-space sums and smooth-PME
        passes go to the workers (the workers own the pairs); everything else is unchanged."""
        import oracle.model as om
        host = self
        saved = (om.pairs, om.realspace, om.spme)
        spme_mod = saved[2]

        class _Pairs:
            def pairs_min_image(self, xyz, box, rc):
                e = np.zeros(0, np.int64)
                return e, e, np.zeros((0, 3))

            def scale_of_pairs(self, I, *a, **k):
                return np.zeros(0)

        class _Real:
            def real_field(self, n, I, J, R, sigma, *args):
                return sum(host.call("real_field", *args))

            def real_dipole_field(self, n, I, J, R, *args):
                return sum(host.call("real_dipole_field", *args))

            def real_forces(self, n, I, J, R, sigma, *args, virial=False):
                parts = host.call("real_forces", *args, virial)
                return tuple(sum(p[k] for p in parts) for k in range(len(parts[0])))

        class _Spme:
            strain_sum = staticmethod(spme_mod.strain_sum)

            def recip_derivs(self, xyz, box, beta, K, order, q, dip, quad, max_order):
                grid = sum(host.call("spread", K, order, q, dip, quad, sliced=(3, 4, 5)))
                phi = spme_mod.convolve(grid, box, K, order, beta)
                parts = host.call("gather", phi, K, order, max_order)
                return [np.concatenate([p[d] for p in parts]) for d in range(max_order + 1)]

        om.pairs, om.realspace, om.spme = _Pairs(), _Real(), _Spme()
        try:
            yield
        finally:
            om.pairs, om.realspace, om.spme = saved

    def _setup(self, s, params):
        self.call("setup", np.asarray(s.xyz, np.float64), np.asarray(s.box, np.float64), params.cutoff,
                  np.asarray(s.excl), s.n)

    def step(self, s, params, tol, outputs=False):
        """One full oracle step for system s; returns (ms, iterations, seconds per stage) and,
        with outputs=True, also (field, dipoles, energy, forces)."""
        from oracle import Oracle
        with self.installed():
            t = {}
            t0 = time.perf_counter()
            self._setup(s, params)
            o = Oracle(s, params)
            t["pairs_and_frames"] = time.perf_counter() - t0
            t1 = time.perf_counter()
            E = o.permanent_field()
            t["field"] = time.perf_counter() - t1
            t1 = time.perf_counter()
            mu, info = o.pcg(E, tol=tol)
            t["pcg"] = time.perf_counter() - t1
            t1 = time.perf_counter()
            energy = o.energy(mu, E)
            F = o.forces(mu)
            t["energy_forces"] = time.perf_counter() - t1
            total = time.perf_counter() - t0
        res = (total * 1e3, info["iters"], {k: round(v, 3) for k, v in t.items()})
        return res + ((E, mu, energy, F),) if outputs else res

    def at_dipoles(self, s, params, mu):
        """The oracle's permanent field, and at the given dipoles the true residual (Debye),
        energy, forces and virial."""
        from oracle import Oracle
        with self.installed():
            self._setup(s, params)
            o = Oracle(s, params)
            E = o.permanent_field()
            resid = o.residual_eps(E - o.apply_A(mu))
            return E, resid, o.energy(mu, E), o.forces(mu), o.virial(mu)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(s, gpu=None):
    """The oracle as it stands, timed on this host: one full step of the 96,000-atom workload
    on every host core (measured, not scaled), and one full step of the 648-atom box on one
    core. With gpu = (field, dipoles, energy, forces, virial) of the library at s (dipoles
    solved to the benchmark's tolerance), also the library's errors against the oracle there:
    field, the true residual of its dipoles, and energy, forces and virial at its dipoles."""
    from oracle import Params
    from paper_2011_01207_gb300 import synth
    cores = host_cores()
    p = Params(beta=BETA, grid=GRID, cutoff=CUTOFF)
    h = HostOracle(cores)
    h.start(s.n)
    errors = None
    try:
        ms, iters, stages = h.step(s, p, TOL)
        if gpu is not None:
            E_g, mu_g, e_g, F_g, V_g = gpu
            E_o, resid, e_o, F_o, V_o = h.at_dipoles(s, p, mu_g)
            rel = lambda a, b: float(np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2)))
            errors = {"err_field_rel_rms": rel(E_g, E_o), "err_true_residual_debye": float(resid),
                      "err_energy_rel": abs(e_g - e_o) / abs(e_o), "err_forces_rel_rms": rel(F_g, F_o),
                      "err_virial_rel_max": float(np.abs(V_g - V_o).max() / np.abs(V_o).max())}
    finally:
        h.stop()
    small = synth.water_box(216, 18.64, 1001)
    p1 = Params(beta=BETA, grid=(24, 24, 24), cutoff=CUTOFF)
    from oracle import Oracle
    t0 = time.perf_counter()
    o = Oracle(small, p1)
    E = o.permanent_field()
    mu, _ = o.pcg(E, tol=TOL)
    o.energy(mu, E)
    o.forces(mu)
    ms1 = (time.perf_counter() - t0) * 1e3
    out = {"value": round(ms, 1), "unit": "ms/step", "cores": cores, "kind": "oracle",
           "sample": f"one full oracle step of the 96,000-atom workload (pairs, frames, permanent field, PCG "
                     f"from alpha E to {TOL} D: {iters} iterations, energy, forces), its pair sums and "
                     f"smooth-PME passes split over {cores} host processes, measured once",
           "cpu": cpu_model(), "stages_s": stages, "oracle_pcg_iters": iters,
           "single_thread_648_atoms_ms_per_step": round(ms1, 1)}
    return out, errors


def run_reference(args):
    """The oracle as it stands on the host cores, on the same workload and metric: every step
    is one full oracle step of the 96,000-atom box at that step's positions (pairs, frames,
    field, PCG from alpha E to 1e-5 D, energy, forces), measured."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import Params
    s = make_system()
    total = args.warmup + args.steps
    traj = trajectory(s, total)
    p = Params(beta=BETA, grid=GRID, cutoff=CUTOFF)
    cores = host_cores()
    h = HostOracle(cores)
    h.start(s.n)
    vals, its, wall = [], [], time.perf_counter()
    try:
        for k in range(total):
            sk = s.copy()
            sk.xyz = traj[k]
            ms, iters, _ = h.step(sk, p, TOL)
            if k >= args.warmup:
                vals.append(ms)
                its.append(iters)
    finally:
        h.stop()
    value = float(np.mean(vals))
    sample = (f"every step one full oracle step of the 96,000-atom box at that step's positions (pairs, frames, "
              f"permanent field, PCG from alpha E to {TOL} D, energy, forces), the oracle's pair sums and "
              f"smooth-PME passes split over {cores} host processes; FP64 NumPy")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ms/step",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(value, 1), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "atoms": s.n, "guess": "plain alpha*E",
                   "pcg_iters_mean": float(np.mean(its))},
        "cpu_baseline": {"value": round(value, 1), "unit": "ms/step", "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": round(value, 1), "unit": "ms/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": round(time.perf_counter() - wall, 1),
    }))


def run_precision(args):
    """Error of every output against the FP64 oracle, in FP64 and in the mixed precision the
    benchmark runs: 648-atom water box, 23,558-atom solvated chain and the 96,000-atom box,
    every atom. Dipoles are solved to the stated tolerance and
    compared with the oracle's solution at 1e-10 D; energy and forces both at the GPU's own
    dipoles (what a user gets) and at the oracle's dipoles (the kernels alone), the virial at
    the oracle's dipoles. The 96,000-atom box is compared in full (the oracle on all host
    cores) at the GPU's dipoles."""
    import torch
    from paper_2011_01207_gb300 import binding, build as _build, synth
    from oracle import Oracle, Params
    _build.build_library()
    debye = 4.80321

    def rel_rms(a, b):
        return float(np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2)))

    cases = [("water_648_atoms_18.64A_grid24", lambda: synth.water_box(216, 18.64, 1001), (24, 24, 24), 1e-6,
              [("fp64", binding.AP_FP64), ("mixed", binding.AP_MIXED), ("fixed", binding.AP_FIXED)]),
             ("chain_23558_atoms_62.2A_grid64", lambda: synth.solvated_chain(2489, 7023, 62.2, 1003), (64, 64, 64), 1e-5,
              [("mixed", binding.AP_MIXED), ("fixed", binding.AP_FIXED)])]
    out = {}
    for name, make, grid, tol, precs in cases:
        s = make()
        o = Oracle(s, Params(beta=BETA, grid=grid, cutoff=CUTOFF))
        E_o = o.permanent_field()
        mu_star, _ = o.pcg(E_o, tol=1e-10)
        e_star, F_star, V_star = o.energy(mu_star, E_o), o.forces(mu_star), o.virial(mu_star)
        for tag, prec in precs:
            c = binding.Context(s, cutoff=CUTOFF, buffer=BUFFER, beta=BETA, grid=grid, precision=prec)
            c.build()
            c.permanent_field()
            info = c.solve(tol=tol, max_iter=200)
            mu = c.mu.cpu().numpy()
            dmu = debye * np.linalg.norm(mu - mu_star, axis=1)
            e, f = c.energy_forces(c.mu)
            e_own, f_own = float(e.cpu()[0]), f.cpu().numpy()
            e, f, V = c.energy_forces(torch.tensor(mu_star, device=c.mu.device), virial=True)
            e_fix, f_fix, V_fix = float(e.cpu()[0]), f.cpu().numpy(), V.cpu().numpy()
            out[f"{name}/{tag}"] = {
                "virial_rel_max_same_dipoles": float(np.abs(V_fix - V_star).max() / np.abs(V_star).max()),
                "atoms": s.n, "pcg_tol_debye": tol, "iterations": info.iterations,
                "field_rel_rms": rel_rms(c.field.cpu().numpy(), E_o),
                "dipole_rms_debye": float(np.sqrt(np.mean(dmu ** 2))), "dipole_max_debye": float(dmu.max()),
                "true_residual_debye": float(o.residual_eps(E_o - o.apply_A(mu))),
                "energy_rel": abs(e_own - e_star) / abs(e_star), "energy_rel_same_dipoles": abs(e_fix - e_star) / abs(e_star),
                "forces_rel_rms": rel_rms(f_own, F_star), "forces_rel_rms_same_dipoles": rel_rms(f_fix, F_star)}
            c.close()
    # AMOEBA's two dipole sets on the same chain, cut into polarization groups
    s, pairs, scales = synth.dp_system(synth.solvated_chain(2489, 7023, 62.2, 1003), 1009)
    o = Oracle(s, Params(beta=BETA, grid=(64, 64, 64), cutoff=CUTOFF), dp=(pairs, scales))
    Ed_o, Ep_o = o.permanent_field_dp()
    mud_star, mup_star, _ = o.pcg_dp(Ed_o, Ep_o, tol=1e-10)
    e_star, F_star = o.energy_dp(mud_star, Ep_o), o.forces_dp(mud_star, mup_star)
    for tag, prec in (("mixed", binding.AP_MIXED), ("fixed", binding.AP_FIXED)):
        c = binding.Context(s, cutoff=CUTOFF, buffer=BUFFER, beta=BETA, grid=(64, 64, 64), precision=prec)
        c.build()
        c.set_scaled_pairs(pairs, scales)
        c.permanent_field_dp()
        info = c.solve_dp(tol=1e-5, max_iter=200)
        mud, mup = c.mu_d.cpu().numpy(), c.mu_p.cpu().numpy()
        dmu = debye * np.linalg.norm(np.concatenate([mud - mud_star, mup - mup_star]), axis=1)
        e, f = c.energy_forces_dp()
        e_own, f_own = float(e.cpu()[0]), f.cpu().numpy()
        e, f = c.energy_forces_dp(torch.tensor(mud_star, device=c.mu.device), torch.tensor(mup_star, device=c.mu.device))
        e_fix, f_fix = float(e.cpu()[0]), f.cpu().numpy()
        out[f"chain_23558_atoms_62.2A_grid64_two_sets/{tag}"] = {
            "atoms": s.n, "pcg_tol_debye": 1e-5, "iterations": info.iterations,
            "field_d_rel_rms": rel_rms(c.field_d.cpu().numpy(), Ed_o),
            "field_p_rel_rms": rel_rms(c.field_p.cpu().numpy(), Ep_o),
            "dipole_rms_debye": float(np.sqrt(np.mean(dmu ** 2))), "dipole_max_debye": float(dmu.max()),
            "true_residual_debye": max(float(o.residual_eps(Ed_o - o.apply_A(mud))),
                                       float(o.residual_eps(Ep_o - o.apply_A(mup)))),
            "energy_rel": abs(e_own - e_star) / abs(e_star), "energy_rel_same_dipoles": abs(e_fix - e_star) / abs(e_star),
            "forces_rel_rms": rel_rms(f_own, F_star), "forces_rel_rms_same_dipoles": rel_rms(f_fix, F_star)}
        c.close()
    # the 96,000-atom box: the full oracle on all host cores (field, and at the GPU's dipoles the
    # true residual, energy, forces and virial)
    s = make_system()
    c = binding.Context(s, cutoff=CUTOFF, buffer=BUFFER, beta=BETA, grid=GRID, precision=binding.AP_MIXED)
    c.build()
    c.permanent_field()
    info = c.solve(tol=TOL, max_iter=200)
    e, f, V = c.energy_forces(c.mu, virial=True)
    E_g, mu_g, e_g, F_g, V_g = (c.field.cpu().numpy(), c.mu.cpu().numpy(), float(e.item()), f.cpu().numpy(),
                                V.cpu().numpy())
    c.close()
    h = HostOracle(host_cores())
    h.start(s.n)
    try:
        E_o, resid, e_o, F_o, V_o = h.at_dipoles(s, Params(beta=BETA, grid=GRID, cutoff=CUTOFF), mu_g)
    finally:
        h.stop()
    out["water_96000_atoms_98.7A_grid100/mixed"] = {
        "atoms": s.n, "pcg_tol_debye": TOL, "iterations": info.iterations, "field_rel_rms": rel_rms(E_g, E_o),
        "true_residual_debye": float(resid), "energy_rel_same_dipoles": abs(e_g - e_o) / abs(e_o),
        "forces_rel_rms_same_dipoles": rel_rms(F_g, F_o),
        "virial_rel_max_same_dipoles": float(np.abs(V_g - V_o).max() / np.abs(V_o).max())}
    print(json.dumps({"metric": "errors against the FP64 oracle", "impl": "ours", "cases": out}))


def run_two_sets(args):
    """AMOEBA's two induced-dipole sets (d and p) on the 23,558-atom solvated chain cut into
    polarization groups: one step = permanent_field_dp + induced_dipoles_pcg_dp (alpha E_d,
    alpha E_p guesses, lockstep to 1e-5 D) + polarization_energy_forces_dp, against the
    single-set step on the same configurations and lists. Also the two-set real-space pair
    kernel against two launches of the single-set one."""
    import torch
    from paper_2011_01207_gb300 import binding, build as _build, synth
    _build.build_library()
    dev = torch.device("cuda", 0)
    s0 = synth.solvated_chain(2489, 7023, 62.2, 1003)
    s, pairs, scales = synth.dp_system(s0, 1009)
    grid = (64, 64, 64)
    total = args.warmup + args.steps
    pos = torch.tensor(trajectory(s, total), device=dev)
    ctx = binding.Context(s, cutoff=CUTOFF, buffer=BUFFER, beta=BETA, grid=grid, precision=binding.AP_MIXED,
                          device=dev)
    ctx.set_scaled_pairs(pairs, scales)
    ctx.xyz.copy_(pos[0])
    ctx.build()
    ctx.permanent_field(out=False)
    tuned = binding.ap_autotune(ctx.ctx, 3)   # launch shapes, untimed set-up
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(k, two):
        xyz = pos[k]
        if k % REBUILD == 0:
            binding.build_neighbour_blocks(ctx.ctx, xyz, ctx.excl_off, ctx.excl_atoms, ctx.n_excl)
        if two:
            binding.permanent_field_dp(ctx.ctx, xyz, ctx.mpole, ctx.frame, ctx.alpha)
            binding.induced_dipoles_pcg_dp(ctx.ctx, None, None, TOL, 200, ctx.mu_d, ctx.mu_p, want_info=False)
            binding.polarization_energy_forces_dp(ctx.ctx, ctx.mu_d, ctx.mu_p, ctx.energy, ctx.forces)
        else:
            binding.permanent_field(ctx.ctx, xyz, ctx.mpole, ctx.frame, ctx.alpha, None)
            binding.induced_dipoles_pcg(ctx.ctx, None, TOL, 200, ctx.mu, want_info=False)
            binding.polarization_energy_forces(ctx.ctx, ctx.mu, ctx.energy, ctx.forces)

    def timed(two):
        ts, its = [], []
        for k in range(args.warmup):
            step(k, two)
        for k in range(args.warmup, total):
            flush.fill_(k & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(k, two)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
            its.append(binding.ap_solve_info_last(ctx.ctx).iterations)
        return float(np.mean(ts)), float(np.mean(its))

    clocks = Clocks(0)
    clocks.start()
    ms2, it2 = timed(True)
    ms1, it1 = timed(False)
    clk = clocks.stop()
    kern = {k: round(binding.ap_time_kernel(ctx.ctx, k, 30), 4) for k in ("real_matvec", "real_matvec2")}
    ctx.close()
    print(json.dumps({
        "metric": "two-set (d/p) polarization step ms, lockstep PCG at 1e-5 D", "impl": "ours",
        "value": round(ms2, 4), "unit": "ms/step", "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": False, "dtype": "f32 pair/PME arithmetic, f64 accumulation", "data": "synthetic",
        "config": {"workload": "chain_23558_atoms_62.2A_grid64_two_sets", "atoms": s.n, "listed_pairs": int(len(pairs)),
                   "iters_mean": it2, "guess": "alpha E_d, alpha E_p",
                   "autotune": {"matvec_ctas_per_sm": tuned[0], "pme_threads": tuned[1]},
                   "single_set": {"ms_per_step": round(ms1, 4), "pcg_iters_mean": it1,
                                  "note": "same configurations and lists, one dipole set"},
                   "l2": "flushed between timed steps (256 MB write)"},
        "kernel_ms": kern,
        "matvec2_vs_two_matvecs": round(kern["real_matvec2"] / (2 * kern["real_matvec"]), 4),
        "clocks": clk}))


KERNEL_WORKLOADS = {
    96000: (32000, 98.7, (100, 100, 100), 1002, "water_96000_atoms_98.7A_grid100_rc7+2_mixed"),
    1065000: (355000, 221.6, (224, 224, 224), 1004, "water_1065000_atoms_221.6A_grid224_rc7+2_mixed"),
}


def run_kernels(args):
    """Every kernel of the path timed alone (CUDA events on its launch stream, warm L2, one
    configuration after one solve from alpha E and one force call), each against its own
    roofline, with the FP32 peak measured on the device. Small enough to run under ncu."""
    import torch
    from paper_2011_01207_gb300 import binding, build as _build, synth
    _build.build_library()
    dev = torch.device("cuda", 0)
    nmol, box, grid, seed, name = KERNEL_WORKLOADS[args.atoms]
    s = synth.water_box(nmol, box, seed)
    ctx = binding.Context(s, cutoff=CUTOFF, buffer=BUFFER, beta=BETA, grid=grid, precision=binding.AP_MIXED,
                          device=dev)
    ctx.build()
    ctx.permanent_field()
    info = ctx.solve(tol=TOL, max_iter=200)
    ctx.energy_forces()
    torch.cuda.synchronize()
    reps = max(1, args.reps)
    kern = {k: binding.ap_time_kernel(ctx.ctx, k, reps) for k in
            ("real_matvec", "spread_dipoles", "gather_field", "convolve", "real_field", "spread_multipoles",
             "pair_forces")}
    ctx.solve(tol=TOL, max_iter=200)
    kern["pcg_vectors"] = binding.ap_time_kernel(ctx.ctx, "pcg_vectors", reps)
    operator_us = {k: round(binding.ap_time_kernel(ctx.ctx, k, reps) * 1e3, 2)
                   for k in ("dipole_operator", "pme_dipoles", "fft_roundtrip")}
    operator_us["pcg_iteration"] = round(pcg_iteration_us(ctx, max(3, reps)), 2)
    fp32, sms = binding.ap_fp32_peak(max(3, reps))
    npairs = pairs_within(s.xyz, s.box, CUTOFF)
    counts = {"real_matvec": info.iterations + 1, "spread_dipoles": info.iterations + 2,
              "gather_field": info.iterations + 1, "convolve": info.iterations + 3, "pcg_vectors": info.iterations}
    kernels = kernel_rooflines(kern, counts, s.n, (s.n + 31) // 32 * 32, npairs, grid, fp32_peak=fp32)
    ctx.close()
    print(json.dumps({"metric": "per-kernel launch time and roofline fraction", "impl": "ours", "workload": name,
                      "atoms": s.n, "pairs_in_cutoff": npairs, "pcg_iters_plain": info.iterations,
                      "fp32_peak_tflops_measured": round(fp32, 2), "sm_count": sms, "reps": reps,
                      "kernels": kernels, "operator_us": operator_us}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline sample")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (resident matvec grid, 128-thread PME kernels)")
    ap.add_argument("--atoms", type=int, default=96000, choices=sorted(KERNEL_WORKLOADS),
                    help="--workload kernels: the 96,000- or the 1,065,000-atom water box")
    ap.add_argument("--reps", type=int, default=20, help="--workload kernels: timed launches per kernel")
    ap.add_argument("--trajectory", default="md", choices=["md", "walk"],
                    help="steps of the water workloads: a real rigid-water MD trajectory (default) or the "
                         "synthetic random walk; the chain workload always walks")
    ap.add_argument("--workload", default="water96k",
                    choices=["water96k", "chain23k", "water1m", "replicas64", "precision", "two_sets", "kernels"],
                    help="water96k: the 96,000-atom box (default); replicas64: 64 uneven replicas in one graph; "
                         "precision: errors of every output against the FP64 oracle; two_sets: AMOEBA's d/p "
                         "dipole sets on the 23,558-atom solvated chain")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "replicas64":
        run_replicas(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "two_sets":
        run_two_sets(args)
    elif args.workload == "kernels":
        run_kernels(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
