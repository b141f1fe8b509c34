"""The oracle's own spread on a run: the reference for comparing runs whose
result depends discontinuously on rounding.

TENO-D's selection (Eqs. 4.7, 4.12) is a threshold on ratios of smoothness
indicators, so near a shock a change of the data at the level of the
arithmetic's rounding can flip a stencil choice; both choices are correct
results of the scheme.  The spread of the FP64 oracle under relative
perturbations of a given size measures how far equally valid runs lie
apart: for the float64 path, perturbations of 1e-15 of the initial state;
for the float32-flux path, perturbations at float32 rounding (1e-7) of the
initial state and, separately, of the state at the start of every step (that
path rounds its reconstruction inputs to float32 on every stage).  A GPU run is then held to a small
multiple of that spread instead of a fixed tolerance."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle as O


def rel_l1(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def _run_perturbed_each_step(P, W0, t_end, rel, rng, max_steps=0):
    """CFL steps to t_end (last one clipped), the state perturbed by
    (1 + rel N(0, 1)) before every step."""
    W = np.array(W0, dtype=np.float64)
    Q = type(P).from_buffer_copy(P)  # the boundary time follows the run
    t, n = 0.0, 0
    while t < t_end and (max_steps <= 0 or n < max_steps):
        W = W * (1 + rel * rng.standard_normal(W.shape))
        dt = min(O.dt(P, W), t_end - t)
        Q.t = P.t + t
        W = O.step(Q, W, dt)
        t += dt
        n += 1
    return W


def fp32_envelope(P, W0, t_end, seeds=(0, 1, 2), max_steps=0):
    """The envelope for the float32-flux path: perturbations of 1e-7 (float32
    rounding) of the initial state, and of the state before every step; the
    larger of the two spreads (a choice sensitive to the initial data at
    float32 level shows only in the first, a drift that rounding feeds on
    every step in the second)."""
    Wa, s_each = oracle_envelope(P, W0, t_end, rel=1e-7, seeds=seeds, max_steps=max_steps, each_step=True)
    _, s_init = oracle_envelope(P, W0, t_end, rel=1e-7, seeds=seeds, max_steps=max_steps)
    return Wa, max(s_each, s_init)


def fp64_envelope(P, W0, t_end, seeds=(0, 1), max_steps=0):
    """The same union for the float64 path, at float64 rounding (1e-15)."""
    Wa, s_each = oracle_envelope(P, W0, t_end, rel=1e-15, seeds=seeds, max_steps=max_steps, each_step=True)
    _, s_init = oracle_envelope(P, W0, t_end, rel=1e-15, seeds=seeds, max_steps=max_steps)
    return Wa, max(s_each, s_init)


def oracle_envelope(P, W0, t_end, rel=1e-15, seeds=(0, 1), max_steps=0, each_step=False):
    """(unperturbed oracle run, max relative-L1 spread of the perturbed runs,
    one per seed): initial state perturbed by (1 + rel N(0, 1)), or with
    each_step the state at the start of every step.  The perturbed runs go in
    threads (the oracle's C calls release the interpreter lock)."""
    Wa = O.run(P, W0, t_end, max_steps=max_steps)[0]

    def one(sd):
        rng = np.random.default_rng(sd)
        if each_step:
            Wb = _run_perturbed_each_step(P, W0, t_end, rel, rng, max_steps)
        else:
            Wb = O.run(P, W0 * (1 + rel * rng.standard_normal(np.shape(W0))), t_end, max_steps=max_steps)[0]
        return rel_l1(Wb, Wa)

    with ThreadPoolExecutor(max_workers=len(seeds)) as ex:
        spreads = list(ex.map(one, seeds))
    return Wa, max(spreads)
