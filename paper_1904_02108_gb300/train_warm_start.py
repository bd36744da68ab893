"""Trains the learned warm start on trajectories the solver itself generates.

    python -m paper_1904_02108_gb300.train_warm_start --out weights.npy \
        [--seeds 8] [--steps 300] [--samples 8192] [--solver cg|mdf]
        [--schedule 24:2e-3,12:5e-4,8:1e-4]

Data: the 256^3 array of 64 propellers with fresh seeds (5000, 5001, ...),
each advanced `steps` steps in tolerance mode (eps <= 1e-4, previous-force
start, with conjugate gradients on the fixed point or, with --solver mdf,
the paper's loop); every step contributes `samples` random points (features
and the target (final du - previous du) / V).  Targets from conjugate
gradients train a network that starts the paper's loop closer to its end
(measured: 122 against 142 iterations per step for targets from the loop
itself on the 256^3 array); neither network shortens conjugate gradients.  Training: Adam on the library's BF16
tensor-core kernels, in stages of (epochs, learning rate), each stage
starting from the previous one's weights.  Writes the FP32 weights (.npy)
and a JSON log beside them.  The stored data/warm_start_256.npy is this
script with its defaults.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--seeds", type=int, default=8)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--samples", type=int, default=8192)
    ap.add_argument("--schedule", default="24:2e-3,12:5e-4,8:1e-4",
                    help="training stages epochs:learning_rate, comma separated")
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--max-iter", type=int, default=1000)
    ap.add_argument("--solver", default="cg", choices=["mdf", "cg"],
                    help="the fixed point's iteration that generates the targets")
    a = ap.parse_args(argv)
    import torch
    from . import binding, learned
    from . import workload as W
    binding.load()
    t0 = time.time()
    ws = [W.dense_array_256(5000 + i) for i in range(a.seeds)]
    X, T = learned.generate(ws, a.steps, tol=a.tol, max_iter=a.max_iter,
                            samples_per_step=a.samples, solver=a.solver)
    t1 = time.time()
    zero_loss = float(0.5 * (T.double() ** 2).sum(1).mean())
    stages = [(int(e), float(lr)) for e, lr in (st.split(":") for st in a.schedule.split(","))]
    P, losses = None, []
    for epochs, lr in stages:
        P, ls = learned.train(X, T, epochs=epochs, batch=a.batch, lr=lr,
                              P0=None if P is None else P.cpu().numpy(),
                              log=lambda m: print(m, flush=True))
        losses += ls
    torch.cuda.synchronize()
    t2 = time.time()
    np.save(a.out, P.cpu().numpy())
    log = {"samples": int(X.shape[0]), "seeds": [5000 + i for i in range(a.seeds)],
           "steps_per_seed": a.steps, "tol": a.tol, "solver": a.solver, "schedule": stages,
           "batch": a.batch,
           "zero_prediction_loss": zero_loss, "losses": losses, "generate_s": t1 - t0,
           "train_s": t2 - t1}
    with open(a.out.rsplit(".", 1)[0] + ".json", "w") as f:
        json.dump(log, f, indent=1)
    print(json.dumps({k: v for k, v in log.items() if k != "losses"}))


if __name__ == "__main__":
    main()
