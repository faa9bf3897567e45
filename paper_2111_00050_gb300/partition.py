"""Sector partition of a space over several GPUs (host-side planning).

Sectors of fixed particle number N and momentum P evolve independently under H
(Sec. III B): the RK4 steps need no data from another sector.  The observables of
Sec. II C-E do: <a_i> pairs a ket of N particles with one of N - 1, <a_i a_j> with
N - 2, <a_i^dag a_j> stays in N.  A partition by contiguous ranges of N therefore
evolves without communication, and at an observation step each rank needs the
amplitudes of the two N-layers just below its range (its halo) from the rank that
holds them; every rank then sums the moments over its own kets, and the sums over
ranks add up to the moments of the whole state.

Nothing here runs on a GPU or moves data; the planner is plain arithmetic over the
sector sizes, and the tests check it with the CPU oracle on two gloo ranks.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence, Tuple


@dataclass
class RankPlan:
    rank: int
    n_lo: int  # first N held
    n_hi: int  # last N held
    sectors: List[int]  # indices into the space's sector list, in order
    halo: List[int]  # sectors of N in [n_lo - 2, n_lo - 1] held by lower ranks
    work: float  # planned work (sum of sector weights)


def plan(sectors: Sequence[Tuple[int, int]], weights: Sequence[float], nranks: int) -> List[RankPlan]:
    """Splits the N-layers of a space (sectors in the order N ascending, then P) into
    `nranks` contiguous ranges of nearly equal work.  weights[s] is the cost of
    sector s (e.g. its dimension times its mean number of terms per ket).  Layers
    are cut at the points where the running work crosses k / nranks of the total
    (a layer is never split: its sectors share the ranking tables and its halo
    would otherwise be on the same rank).  Ranks beyond the number of layers get
    empty ranges."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    if len(sectors) != len(weights):
        raise ValueError("one weight per sector")
    layers = sorted({N for N, _ in sectors})
    layer_work = {N: 0.0 for N in layers}
    for (N, _), w in zip(sectors, weights):
        layer_work[N] += float(w)
    total = sum(layer_work.values())
    cuts = []  # first layer index of ranks 1 .. nranks-1
    run, k = 0.0, 1
    for i, N in enumerate(layers):
        # close rank k-1 before layer i when adding it would overshoot its share by
        # more than stopping short does
        while k < nranks and i > 0 and run + layer_work[N] / 2 > k * total / nranks:
            cuts.append(i)
            k += 1
        run += layer_work[N]
    while len(cuts) < nranks - 1:
        cuts.append(len(layers))
    bounds = [0] + cuts + [len(layers)]
    plans = []
    for r in range(nranks):
        held = layers[bounds[r]:bounds[r + 1]]
        if held:
            lo, hi = held[0], held[-1]
        else:  # an empty rank: an empty range above every layer
            lo, hi = (layers[-1] + 1 if layers else 0), (layers[-1] if layers else -1)
        own = [s for s, (N, _) in enumerate(sectors) if lo <= N <= hi]
        halo = [s for s, (N, _) in enumerate(sectors) if lo - 2 <= N < lo] if held else []
        plans.append(RankPlan(r, lo, hi, own, halo, sum(weights[s] for s in own)))
    return plans


def owner_of_layer(plans: Sequence[RankPlan], N: int) -> int:
    """Rank whose range holds particle number N (-1 if none)."""
    for p in plans:
        if p.n_lo <= N <= p.n_hi:
            return p.rank
    return -1
