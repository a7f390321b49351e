"""Checkpoint and resume of a minSR run (host-side state only).

One step of Algorithm 1 is a function of theta, the momentum m (App. B),
the step index t (learning-rate decay, Tab. I, and the Philox counter of
the sampler), the hyper-parameters (the Philox key among them) and, with
Levenberg-Marquardt damping (App. G), the damping the context holds on the
device, which every step reports as stats.lambda_next.  save() writes these;
load() restores them into a context of the same model, Hamiltonian and
precision, after which the run continues bit for bit.
"""
import dataclasses
import json

import numpy as np
import torch

from . import nqs
from .inputs import HParams


def save(path, theta, mom, next_step, hp: HParams, stats, damping_omega=0.0):
    """Write theta, m, the index of the next step, hp, the damping factor
    (0: off) and the damping of the next step (stats of the last step)."""
    d = nqs.decode_stats(stats)
    np.savez(path, theta=theta.detach().cpu().numpy(), mom=mom.detach().cpu().numpy(),
             next_step=np.int64(next_step), damping_omega=np.float64(damping_omega),
             lambda_next=np.float64(d["lambda_next"]), hp=json.dumps(dataclasses.asdict(hp)))


def load(path, ctx):
    """theta and m on ctx's device, the index of the next step and hp; sets
    the context's damping to the saved state (on at the saved damping, or
    off)."""
    z = np.load(path)
    hp = HParams(**json.loads(str(z["hp"])))
    theta = torch.tensor(z["theta"], dtype=torch.float64, device=ctx.device)
    mom = torch.tensor(z["mom"], dtype=torch.float64, device=ctx.device)
    omega = float(z["damping_omega"])
    # always set: a saved run without damping switches off damping the
    # target context may have on (omega <= 1 turns it off)
    ctx.set_damping(omega, float(z["lambda_next"]) if omega > 1.0 else 0.0)
    return theta, mom, int(z["next_step"]), hp
