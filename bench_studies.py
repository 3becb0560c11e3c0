"""Experiments beside the bench line (``bench.py --study NAME``): the paper's
energy traces and 50-shot statistics at its QUBO sizes (Fig. 2-4), the fixed
c0 against a scan (section "Results"), schedule learning through the adjoint,
the adjoint's cost, the QUBO build on host and GPU, and every step kernel on
one workload. Each prints JSON lines; ``--record FILE`` also writes them, with
the command that made them, to FILE (markdown)."""
import json
import os
import sys
import time

import numpy as np


class Recorder:
    def __init__(self, path, argv):
        self.path = path
        self.lines = []
        self.cmd = "python bench.py " + " ".join(a for a in argv if not a.startswith("--record")
                                                and a != path)

    def emit(self, rec):
        s = json.dumps(rec)
        print(s, flush=True)
        self.lines.append(s)

    def close(self, title):
        if not self.path:
            return
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        with open(self.path, "w") as f:
            f.write(f"# {title}\n\nCommand (on one GB300):\n\n```\n{self.cmd}\n```\n\n"
                    f"Records (one JSON object per line):\n\n```\n")
            f.write("\n".join(self.lines))
            f.write("\n```\n")


def _trace(sb, ctx, variant, a0, c0, dt, S, R, seed, every, stream, dev):
    """Energies of all R shots every `every` steps and the time to each checkpoint."""
    import torch
    sched = torch.tensor(np.array([a0 * k / (S - 1) for k in range(S)], np.float32), device=dev)
    d_E = torch.empty(R, dtype=torch.float64, device=dev)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)
    sb.sb_run(ctx, variant, a0, c0, dt, 0, R, seed, None, stream)
    t0 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    marks, Es = [], []
    for k0 in range(0, S, every):
        n = min(every, S - k0)
        sb.sb_advance(ctx, variant, a0, c0, dt, n, sched[k0:k0 + n], stream)
        sb.sb_readout_device(ctx, d_E, None, None, None, stream)
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        marks.append(e)
        Es.append(d_E.clone())
    torch.cuda.synchronize(dev)
    return [t0.elapsed_time(m) * 1e-3 for m in marks], [e.cpu().numpy() for e in Es]


def _event(sb, spec):
    ev = sb.sb_event_generate(spec["seed"], sb.event_params(n_tracks=spec["n_tracks"],
                                                            noise_frac=spec["noise_frac"]))
    return ev, sb.sb_qubo_build(ev, sb.build_params(**spec["cuts"]))


def _us_per_step(sb, ctx, variant, R, S, stream, dev, reps=2):
    import torch
    sched = torch.tensor(np.linspace(0, 1, S).astype(np.float32), device=dev)
    sb.sb_run(ctx, variant, 1.0, 0.0, 0.5, 0, R, 7, None, stream)
    sb.sb_advance(ctx, variant, 1.0, 0.0, 0.5, S, sched, stream)
    sb.sb_advance(ctx, variant, 1.0, 0.0, 0.5, S, sched, stream)
    torch.cuda.synchronize(dev)
    best = 1e30
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sb.sb_advance(ctx, variant, 1.0, 0.0, 0.5, S, sched, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        best = min(best, e0.elapsed_time(e1) * 1e3 / S)
    return best


def run_study(args):
    import torch
    import bench
    import paper_2402_14718_gb300 as sb
    from paper_2402_14718_gb300.workloads import CUTS_DENSE, PAPER_SIZES, WORKLOADS
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream(dev)
    rec = Recorder(args.record, sys.argv[1:])
    if args.study == "kernels":
        # every step form on one workload: microseconds per step (graph replay,
        # CUDA events, best of 2 runs of the S-step schedule), the HBM roofline fraction of the
        # method's bytes, and whether the state equals the first form's
        w = bench.workload(args.workload, 0, args.variant)
        pairs = bench.build_events(sb, w)
        qs = [q for _, q in pairs]
        R = w["R"]
        N = sum(q.n for q in qs)
        nnz = sum(q.nnz for q in qs)
        prec = sb.SB_J_BF16 if w["jprec"] == "bf16" else sb.SB_J_FP32
        S = w["S"]   # the workload's whole schedule: the spins' wall occupancy changes the cost
        hbm, _ = bench.peaks()
        alg = 16 * N * R + nnz * (6 if prec == sb.SB_J_BF16 else 8) + 8 * N
        forms = [("plain, untiled", False, [(sb.SB_OPT_ROWS_PER_WARP, 0)]),
                 ("plain, row groups of 2", False, [(sb.SB_OPT_ROWS_PER_WARP, 2)]),
                 ("plain, tiled", False, [(sb.SB_OPT_TILED, 1), (sb.SB_OPT_ROWS_PER_WARP, 0)]),
                 ("plain, bulk-copy ring", False, [(sb.SB_OPT_STREAM, 1)]),
                 ("factored", True, []),
                 ("factored, dedicated kernel", True, [(sb.SB_OPT_ROWS_PER_WARP, 0)])]
        if w["variant"] == "dsb":
            forms = [("plain, sign bytes", False, []),
                     ("plain, FP32 positions", False, [(sb.SB_OPT_DSB_SIGNS, 0)]),
                     ("factored, sign bytes", True, [])]
        ref = None
        for name, factor, opts in forms:
            ctx = bench.make_ctx(sb, qs, prec, factor=factor)
            for k, v in opts:
                sb.sb_set_option(ctx, k, v)
            us = _us_per_step(sb, ctx, w["variant"], R, S, stream, dev)
            x, y = sb.sb_get_state(ctx)
            same = None
            if ref is None:
                ref = (x, y)
            else:
                same = bool(np.array_equal(ref[0], x) and np.array_equal(ref[1], y))
            rec.emit({"study": "kernels", "workload": w["name"], "variant": w["variant"], "N": N,
                      "nnz": nnz, "R": R, "form": name, "us_per_step": us,
                      "hbm_frac": alg / (us * 1e-6) / 1e9 / hbm,
                      "same_state_as_first": same,
                      "factor": sb.sb_factor_info(ctx) if factor else None})
            sb.sb_destroy(ctx)
        rec.close(f"Step forms on {w['name']} ({w['variant']})")
        return 0
    if args.study == "paper-sizes":
        # section "Results": a0 = dt = 1, fixed c0, 50 shots; bSB and dSB
        S, R, every = (args.sb_steps or 2000), 50, 20
        for p in PAPER_SIZES:
            ev = sb.sb_event_generate(p["seed"], sb.event_params(n_tracks=p["n_tracks"]))
            q = sb.sb_qubo_build(ev, sb.build_params(**CUTS_DENSE))
            ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, sb.SB_J_BF16)
            off = sb.sb_info(ctx)["offset"]
            for variant in ("bsb", "dsb"):
                times, Es = _trace(sb, ctx, variant, 1.0, 0.0, 1.0, S, R, 1, every, stream, dev)
                fin = Es[-1]
                T, Eb, _ = sb.sb_best(ctx)
                sc = sb.sb_tracks(ev, q, T)
                pick = [int(v) for v in np.linspace(0, len(Es) - 1, 12)]
                rec.emit({
                    "study": "paper-sizes", "paper_N": p["paper_N"], "N": q.n, "nnz": q.nnz,
                    "tracks": p["n_tracks"], "variant": variant, "shots": R, "steps": S,
                    "a0": 1.0, "dt": 1.0, "c0": "auto",
                    "final_ising_min": float(fin.min() - off), "final_ising_mean": float(fin.mean() - off),
                    "final_ising_std": float(fin.std()), "final_ising_max": float(fin.max() - off),
                    "run_seconds": times[-1],
                    "trace": [{"t": times[i], "step": int((i + 1) * every), "mean": float(Es[i].mean() - off),
                               "min": float(Es[i].min() - off), "max": float(Es[i].max() - off)}
                              for i in pick],
                    "efficiency": sc["efficiency"], "purity": sc["purity"]})
        rec.close("Energy traces and 50-shot statistics at the paper's QUBO sizes (Fig. 2-4)")
        return 0
    if args.study == "adjoint":
        # 500-track workload: bSB forward vs sb_backward (checkpoint every 32 steps)
        ev, q = _event(sb, dict(seed=WORKLOADS["event500"]["seed"], n_tracks=500,
                                noise_frac=0.1, cuts=WORKLOADS["event500"]["cuts"]))
        w = WORKLOADS["event500"]
        ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, sb.SB_J_FP32)
        sb.sb_set_weights(ctx, q.cls, q.quality, 1.0, 1.0)
        S, R, c0 = (args.sb_steps or w["steps"]), w["replicas"], sb.sb_info(ctx)["c0_auto"]
        sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)   # both directions launch one kernel per step
        sb.sb_run(ctx, "bsb", 1.0, c0, 0.5, S, R, 1, None, stream)
        sb.sb_backward(ctx, 1.0, c0, 0.5, S, R, 1, None, 32)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(3):
            sb.sb_run(ctx, "bsb", 1.0, c0, 0.5, S, R, 1, None, stream)
        torch.cuda.synchronize(dev)
        t_fwd = (time.perf_counter() - t0) / 3
        for K in (32, S):   # checkpoint every 32 steps; whole run recorded once
            sb.sb_backward(ctx, 1.0, c0, 0.5, S, R, 1, None, K)
            t0 = time.perf_counter()
            for _ in range(3):
                loss, g = sb.sb_backward(ctx, 1.0, c0, 0.5, S, R, 1, None, K)
            t_bwd = (time.perf_counter() - t0) / 3
            rec.emit({"study": "adjoint", "N": q.n, "R": R, "steps": S, "ckpt_every": K,
                      "forward_s": t_fwd, "backward_s": t_bwd,
                      "backward_over_forward": t_bwd / t_fwd, "loss": loss, "grads": g})
        rec.close("Adjoint (sb_backward) against the forward run, 500-track event")
        return 0
    if args.study == "build":
        # QUBO construction time (left out of the paper's timings): host C++ vs GPU
        for name in ("event1000", "event10k"):
            w = WORKLOADS[name]
            ev = sb.sb_event_generate(w["seed"], sb.event_params(n_tracks=w["n_tracks"],
                                                                 noise_frac=w["noise_frac"]))
            p = sb.build_params(**w["cuts"])
            t0 = time.perf_counter()
            qh = sb.sb_qubo_build(ev, p)
            t_host = time.perf_counter() - t0
            sb.sb_qubo_build_device(ev, p)                     # warm-up
            t0 = time.perf_counter()
            qd, ms = sb.sb_qubo_build_device(ev, p)
            t_dev = time.perf_counter() - t0
            rec.emit({"study": "build", "workload": name, "N": qh.n, "nnz": qh.nnz,
                      "host_s": t_host, "device_kernels_ms": ms, "device_call_s": t_dev,
                      "same_structure": bool(qd.n == qh.n and np.array_equal(qd.col, qh.col))})
        rec.close("QUBO build: host C++ against the GPU builder")
        return 0
    if args.study == "c0-scan":
        # section "Results": fixed c0 versus a scan
        w = WORKLOADS["event1000"]
        ev = sb.sb_event_generate(w["seed"], sb.event_params(n_tracks=w["n_tracks"],
                                                             noise_frac=w["noise_frac"]))
        q = sb.sb_qubo_build(ev, sb.build_params(**w["cuts"]))
        ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, sb.SB_J_BF16)
        part = ev.arrays()["particle"]
        truth = np.array([1 if part[a] == part[b] == part[c] >= 0 else 0 for a, b, c in q.trip],
                         np.int8)
        E_truth = float(sb.sb_energy(ctx, np.where(truth > 0, 1, -1).astype(np.int8)[:, None])[0, 0])
        c0a = sb.sb_info(ctx)["c0_auto"]
        S, R = 2000, 64
        for variant in ("bsb", "dsb"):
            for f in (0.25, 0.5, 1.0, 2.0, 3.0, 4.0):
                sb.sb_run(ctx, variant, 1.0, -f, 0.5, S, R, 3, None, stream)
                E = sb.sb_energy(ctx, None, R)[0]
                T, _, _ = sb.sb_best(ctx)
                sc = sb.sb_tracks(ev, q, T)
                rec.emit({"study": "c0-scan", "variant": variant, "c0": c0a * f, "c0_over_auto": f,
                          "median_E": float(np.median(E)), "min_E": float(E.min()),
                          "E_truth": E_truth, "efficiency": sc["efficiency"], "purity": sc["purity"]})
        rec.close("c0 scan on the 1000-track event (section \"Results\": fixed c0 against a scan)")
        return 0
    if args.study == "schedule":
        # a(t) learned by gradient descent on the mean relaxed energy (sb_backward)
        w = WORKLOADS["event500"]
        ev = sb.sb_event_generate(w["seed"], sb.event_params(n_tracks=w["n_tracks"],
                                                             noise_frac=w["noise_frac"]))
        q = sb.sb_qubo_build(ev, sb.build_params(**w["cuts"]))
        ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, sb.SB_J_FP32)
        sb.sb_set_weights(ctx, q.cls, q.quality, 1.0, 1.0)
        # the relaxed energy at the last step is piecewise constant in a(t) once every
        # spin sits on a wall (long bSB runs): learn on a horizon that ends mid-bifurcation
        S, R, c0 = (args.sb_steps or 60), w["replicas"], sb.sb_info(ctx)["c0_auto"]
        a = torch.tensor(np.array([0.5 * k / (S - 1) for k in range(S)], np.float32), device=dev)
        g = torch.zeros(S, dtype=torch.float64, device=dev)
        for it in range(args.steps):
            loss, grads = sb.sb_backward(ctx, 1.0, c0, 0.5, S, R, 11, a, 32, g)
            sb.sb_run(ctx, "bsb", 1.0, c0, 0.5, S, R, 11, a, stream)
            E = sb.sb_energy(ctx, None, R)[0]
            x, _ = sb.sb_get_state(ctx)
            rec.emit({"study": "schedule", "iter": it, "steps": S, "relaxed_loss": loss,
                      "fraction_on_walls": float(np.mean(np.abs(x) == 1.0)),
                      "median_qubo_E": float(np.median(E)), "min_qubo_E": float(E.min()),
                      "grad_inf": float(g.abs().max()), "dL_ddt": grads["dt"],
                      "dL_dc0": grads["c0"]})
            step = 0.05 * g / max(float(g.abs().max()), 1e-30)
            a = torch.clamp(a - step.to(torch.float32), 0.0, 1.0).contiguous()
        rec.close("Schedule a(t) learned through the adjoint, 500-track event")
        return 0
    return 0
