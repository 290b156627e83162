"""Seeded synthetic workloads for the serving loop and the batched advance.

Only workload descriptions live here (grids, bond dimensions, temperature settings, arrival
times); none of the method's arithmetic.  The mixes follow the paper's parameter study of the
2D TFIM (J = -1, h = 2, dt = 0.25; the three initial-state temperatures of Eq. initial_state)
and the grid sizes of its Table of simulated lattices, at bond dimensions that fit one GPU.
"""
import math

import numpy as np

# the three temperature settings of the initial product state: offset of theta above theta_min
TEMPERATURE_DTHETA = {"low": 0.0, "mid": 2.0 * math.pi / 9.0, "high": 3.0 * math.pi / 9.0}

SERVE_GRIDS = ((4, 4), (5, 6), (6, 6), (6, 8), (7, 8))
SERVE_CHIS = (64, 256, 1024)


def serving_jobs(count, rate, seed, grids=SERVE_GRIDS, chis=SERVE_CHIS, steps=20, order=2, prec="split_bf16x3",
                 J=-1.0, h=2.0, dt=0.25):
    """`count` jobs arriving as a Poisson stream of mean `rate` per second (seeded).

    Each job draws its grid and bond dimension uniformly from the given lists and its
    temperature setting uniformly from low / mid / high.  Arrival times are in seconds from 0.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    arrivals = np.cumsum(gaps) - gaps[0]
    names = sorted(TEMPERATURE_DTHETA)
    jobs = []
    for i in range(count):
        Lx, Ly = grids[int(rng.integers(len(grids)))]
        temp = names[int(rng.integers(len(names)))]
        jobs.append(dict(jid=i, arrival=float(arrivals[i]), Lx=Lx, Ly=Ly, chi=int(chis[int(rng.integers(len(chis)))]),
                         temperature=temp, dtheta=TEMPERATURE_DTHETA[temp], J=J, h=h, dt=dt, steps=steps,
                         order=order, prec=prec, seed=int(rng.integers(1 << 31))))
    return jobs


def batched_mix(count, seed, grids=((4, 4), (4, 6), (5, 6), (6, 6)), chis=(32, 64, 128, 256, 512), prec="fp32"):
    """`count` independent MPS of uneven grid and bond dimension, with the initial-state offset
    dtheta drawn uniformly in [pi/12, pi/3] (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        Lx, Ly = grids[int(rng.integers(len(grids)))]
        out.append(dict(jid=i, Lx=Lx, Ly=Ly, chi=int(chis[int(rng.integers(len(chis)))]),
                        dtheta=float(rng.uniform(math.pi / 12, math.pi / 3)), J=-1.0, h=2.0, dt=0.25, order=2,
                        prec=prec, seed=int(rng.integers(1 << 31))))
    return out
