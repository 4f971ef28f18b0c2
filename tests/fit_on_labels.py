"""Fit of the neural GCDF on labelled samples of the capsule robot's GCDF, and
the trained field's properties (Sec. III-C training, Table I losses, Eq. 9
total loss; Theorem 1; Sec. V-A single-step projection test).

The training data come from the FP64 oracle (``oracle.labels``: points on
height levels, dense zero-level subsets moved by translation, Eq. 5-8); the
network, its gradients and every training step run in libgcdf's kernels
through the autograd Function ``field_grad`` (BF16 tensor-core GEMMs with FP32
master weights, or FP32).  This file is test infrastructure: the GPU test
imports it with a small configuration, and run as a script it performs the
full experiment and prints one JSON record:

    python tests/fit_on_labels.py [--points 4096 --zero 4096 --steps 1500 ...]

Losses (Table I, hat = label): L_dist = mean (f^ - f)^2;
L_grad = mean (1 - cos(grad f^, grad f))^2; L_eikonal = mean (||grad f||_{M^-1} - 1)^2;
L_tension = mean ||grad f||^2; L = 5 L_dist + 0.1 L_grad + 0.01 L_eik + 0.01 L_tension
(the weights of Sec. V-A).  M = I.  Adam, the learning rate halved at 50 %
and 75 % of the steps (the paper halves it without giving the schedule).

Trained-field properties, on held-out points:
  * the four losses;
  * ||grad_q f||_{M^-1} off the nonsmooth set (labels whose two nearest
    zero-level samples differ by more than `gap_min` and |f^| > 0.05), which
    Theorem 1 fixes at 1;
  * the single-step projection q+ = q - f M^-1 grad_q f (gcdf_project on the
    trained weights) from random initial configurations towards target
    points, scored by the residual ratio |f_s(p, q+)| / |f_s(p, q0)| of the
    exact capsule SDF (the test of Sec. V-A).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

SHAPE = (10, 512, 5)
LAMBDA = (5.0, 0.1, 0.01, 0.01)


def make_data(points, per_point, zero, heights, seed, workers, p_radius=3.0):
    """(q, p, f, grad, gap) FP64 from the oracle (spawned worker pool)."""
    from oracle import labels
    return labels.generate(10, points, per_point, zero, p_radius, seed, workers, n_heights=heights)


def table1_losses(torch, f, dq, f_hat, g_hat, m_inv=None):
    """The four Table I terms (tensors) for predicted (f, dq) and labels."""
    l_dist = ((f_hat - f) ** 2).mean()
    cos = (g_hat * dq).sum(1) / (g_hat.norm(dim=1) * dq.norm(dim=1) + 1e-12)
    l_grad = ((1.0 - cos) ** 2).mean()
    nrm = dq.norm(dim=1) if m_inv is None else torch.sqrt((dq * dq * m_inv).sum(1))
    l_eik = ((nrm - 1.0) ** 2).mean()
    l_ten = (dq * dq).sum(1).mean()
    return l_dist, l_grad, l_eik, l_ten


def train(g, torch, data, steps, batch, lr, precision="bf16", seed=0, log_every=0):
    """Adam on the Table I / Eq. 9 loss; returns (weights, history)."""
    q, p, f_hat, g_hat = (torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda() for x in data[:4])
    S = q.shape[0]
    w = torch.from_numpy(synth.he_uniform_weights(synth.NetShape(*SHAPE), seed)).cuda().requires_grad_(True)
    opt = torch.optim.Adam([w], lr=lr)
    sched = torch.optim.lr_scheduler.MultiStepLR(opt, [steps // 2, (3 * steps) // 4], 0.5)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    perm, pos, hist = torch.randperm(S, device="cuda", generator=gen), 0, []
    for it in range(steps):
        if pos + batch > S:
            perm, pos = torch.randperm(S, device="cuda", generator=gen), 0
        idx = perm[pos: pos + batch]
        pos += batch
        qb, pb = q[idx].contiguous(), p[idx].contiguous()
        opt.zero_grad()
        f, dq = g.field_grad(w, qb, pb, SHAPE, precision=precision)
        parts = table1_losses(torch, f, dq, f_hat[idx], g_hat[idx])
        loss = sum(lam * x for lam, x in zip(LAMBDA, parts))
        loss.backward()
        opt.step()
        sched.step()
        if log_every and (it % log_every == 0 or it == steps - 1):
            hist.append([it] + [float(x.detach()) for x in parts])
    return w.detach(), hist


def evaluate(g, torch, w, data, gap_min=0.05, precision="fp32"):
    """Table I losses on (q, p, f^, grad f^, gap) and ||grad f|| statistics off
    the nonsmooth set."""
    q, p, f_hat, g_hat = (torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda() for x in data[:4])
    f, dq = g.fit_value_grad(SHAPE, w, q, p, precision=precision)
    parts = [float(x) for x in table1_losses(torch, f, dq, f_hat, g_hat)]
    nrm = dq.norm(dim=1).cpu().numpy()
    smooth = (np.asarray(data[4]) > gap_min) & (np.abs(np.asarray(data[2])) > 0.05)
    n_s = nrm[smooth]
    return {"L_dist": parts[0], "L_grad": parts[1], "L_eikonal": parts[2], "L_tension": parts[3],
            "samples": int(q.shape[0]),
            "grad_norm_off_nonsmooth": {"samples": int(n_s.size), "mean": float(n_s.mean()),
                                        "std": float(n_s.std()), "p5": float(np.percentile(n_s, 5)),
                                        "p95": float(np.percentile(n_s, 95))},
            "label_f_mean": float(np.mean(data[2])), "abs_err_f_mean": float(np.abs(f.cpu().numpy() - data[2]).mean())}


def projection_test(g, torch, w, n_targets=128, n_inits=128, half_range=2.0, seed=5):
    """Sec. V-A: targets uniform in [-r, r]^2 x [0, 2] around a base at the
    origin, initial configurations with the base at the origin and yaw / joints
    uniform in [-pi, pi]; one projection step through the trained field
    (gcdf_project, FP32 path) and the residual ratio of the exact SDF."""
    from oracle import robot as R
    arm = R.mobile_arm_7()
    rng = synth.SplitMix64(seed)
    P = synth.uniform_points(rng, n_targets, [-half_range, -half_range, 0.0], [half_range, half_range, 2.0])
    N = n_targets * n_inits
    q0 = np.zeros((N, 10))
    q0[:, 2:] = rng.uniform(N * 8, -math.pi, math.pi).reshape(N, 8)
    tgt = np.repeat(np.arange(n_targets), n_inits).astype(np.int32)
    net = g.create_net(*SHAPE, w.cpu().numpy(), "fp32")
    qd = torch.from_numpy(q0.astype(np.float32)).cuda()
    pd = torch.from_numpy(P.astype(np.float32)).cuda()
    off = torch.arange(N + 1, device="cuda", dtype=torch.int32)
    idx = torch.from_numpy(tgt).cuda()
    qp = g.project(net, qd, pd, part_offsets=off, part_idx=idx).cpu().numpy().astype(np.float64)
    r0 = np.empty(N)
    r1 = np.empty(N)
    for t in range(n_targets):
        sl = slice(t * n_inits, (t + 1) * n_inits)
        r0[sl] = np.abs(R.sdf_batch(arm, P[t], q0[sl]))
        r1[sl] = np.abs(R.sdf_batch(arm, P[t], qp[sl]))
    ratio = r1 / np.maximum(r0, 1e-12)
    return {"targets": n_targets, "inits_per_target": n_inits, "target_box_m": half_range,
            "residual_ratio": {"median": float(np.median(ratio)), "mean": float(ratio.mean()),
                               "p10": float(np.percentile(ratio, 10)), "p90": float(np.percentile(ratio, 90)),
                               "frac_below_0.1": float((ratio < 0.1).mean()),
                               "frac_below_0.5": float((ratio < 0.5).mean())},
            "initial_abs_sdf_mean": float(r0.mean()), "projected_abs_sdf_mean": float(r1.mean())}


def run(points=4096, per_point=256, zero=4096, heights=64, held_points=128, steps=1500, batch=65536,
        lr=2e-3, precision="bf16", workers=None, log_every=100, seed=0):
    import torch
    import __graft_entry__
    workers = workers or os.cpu_count() or 8
    t0 = time.time()
    data = make_data(points + held_points, per_point, zero, heights, seed, workers)
    t_lab = time.time() - t0
    cut = points * per_point
    tr = tuple(x[:cut] for x in data)
    ho = tuple(x[cut:] for x in data)
    __graft_entry__.build()
    import paper_2601_18548_gb300 as g
    w0 = torch.from_numpy(synth.he_uniform_weights(synth.NetShape(*SHAPE), seed)).cuda()
    before = evaluate(g, torch, w0, ho)
    torch.cuda.synchronize()
    t1 = time.time()
    w, hist = train(g, torch, tr, steps, min(batch, cut), lr, precision, seed, log_every)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    assert g.fit_device_status() == 0
    after = evaluate(g, torch, w, ho)
    proj = projection_test(g, torch, w)
    proj0 = projection_test(g, torch, w0)
    return {"experiment": "fit on oracle labels", "net": "10-DOF 5 x 512 SiLU", "precision": precision,
            "labels": {"train_samples": cut, "held_out_samples": int(held_points * per_point),
                       "points": points, "per_point": per_point, "height_levels": heights,
                       "zero_lines_per_level": zero, "seconds": t_lab, "workers": workers},
            "training": {"steps": steps, "batch": min(batch, cut), "lr": lr, "lambda": LAMBDA,
                         "seconds": t_train, "ms_per_step": 1e3 * t_train / max(steps, 1),
                         "history": hist},
            "held_out_before": before, "held_out_after": after,
            "projection_trained": proj, "projection_untrained": proj0}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--points", type=int, default=4096)
    ap.add_argument("--per-point", type=int, default=256)
    ap.add_argument("--zero", type=int, default=4096)
    ap.add_argument("--heights", type=int, default=64)
    ap.add_argument("--held-points", type=int, default=128)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--workers", type=int, default=None)
    a = ap.parse_args(argv)
    out = run(a.points, a.per_point, a.zero, a.heights, a.held_points, a.steps, a.batch, a.lr, a.precision,
              a.workers)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
