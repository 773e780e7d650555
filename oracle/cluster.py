"""CPU oracle of the paper's parallel merging clustering (TEST INFRASTRUCTURE
ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU baseline may use it;
the product path never does, and it shares no code with the CUDA kernels).

What it computes, in the paper's order (Sec. "Parallel Merging Algorithm"
and "Merging Criterion", Eq. 1, Eq. 2, the phi equation, Table 1):

  * every pixel starts as a region whose ID is its linear index; its
    homogeneity descriptor is w = (z, phi) with phi = arctan(d sqrt(I))
    (d the radial distance, I the intensity, z the distance along the
    optical axis);
  * one synchronous round: every region looks at its 4-neighbourhood
    neighbour regions S, keeps those with |z_R - z_S| <= t_z and
    |phi_R - phi_S| <= t_phi (Eq. 1), and picks the one minimising
    f = alpha_z |z_R - z_S| + alpha_phi |phi_R - phi_S| (Eq. 2), ties going
    to the larger ID;
  * two regions merge only when the choice is mutual; the merged region
    takes the greater ID and its descriptor is the mean over all its pixels
    (running sums of z and phi divided by the pixel count);
  * rounds repeat until no region has a qualifying neighbour.

Readings: the "mean average of both regions" is the mean over the merged
region's pixels (z_R is defined as the region's average distance); every
decision (criterion, f, ties, the means it compares) is taken in FP32 with
the operations rounded one at a time, as the kernel takes them; phi is the
FP64 arctan of the FP32 inputs rounded to FP32.

Vectorised numpy; ``brute()`` is an independent loop-by-loop version for
tiny grids.
"""
from __future__ import annotations

import numpy as np

# Table 1 of the paper, rounded to FP32
T_Z = np.float32(0.04)
T_PHI = np.float32(0.009)
ALPHA_Z = np.float32(8.0 / np.pi)
ALPHA_PHI = np.float32(4.0 / 3.0)


def phi(d, intensity):
    """phi = arctan(d sqrt(I)) in FP64 from the FP32 inputs, rounded to FP32."""
    d64 = np.asarray(d, np.float32).astype(np.float64)
    i64 = np.asarray(intensity, np.float32).astype(np.float64)
    return np.arctan(d64 * np.sqrt(i64)).astype(np.float32)


def _f32(x):
    return np.asarray(x, dtype=np.float32)


def cluster(z, d, intensity, t_z=T_Z, t_phi=T_PHI, alpha_z=ALPHA_Z, alpha_phi=ALPHA_PHI, max_rounds=None):
    """One (h, w) frame.  Returns (labels (h, w) int32, rounds, region counts
    per round, mean_z, mean_phi, size) -- the last three indexed by region ID
    (size 0 for IDs that merged away)."""
    z = _f32(z)
    h, w = z.shape
    n = h * w
    t_z, t_phi, a_z, a_phi = (np.float32(v) for v in (t_z, t_phi, alpha_z, alpha_phi))
    ph = phi(d, intensity).reshape(n)
    sum_z, sum_p = z.reshape(n).copy(), ph.copy()
    mean_z, mean_p = sum_z.copy(), sum_p.copy()
    size = np.ones(n, np.int64)
    label = np.arange(n, dtype=np.int64)
    idx = np.arange(n).reshape(h, w)
    # pixel pairs of the 4-neighbourhood (each unordered pair once)
    pa = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    pb = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    counts = [n]
    rounds = 0
    limit = n if max_rounds is None else max_rounds
    while rounds < limit:
        R, S = label[pa], label[pb]
        keep = R != S
        R, S = R[keep], S[keep]
        if R.size == 0:
            break
        # unordered region pairs, each once
        lo, hi = np.minimum(R, S), np.maximum(R, S)
        pairs = np.unique(np.stack([lo, hi], axis=1), axis=0)
        lo, hi = pairs[:, 0], pairs[:, 1]
        dz = np.abs(mean_z[lo] - mean_z[hi])           # FP32, rounded once each
        dp = np.abs(mean_p[lo] - mean_p[hi])
        ok = (dz <= t_z) & (dp <= t_phi)               # Eq. 1
        if not ok.any():
            break
        lo, hi, dz, dp = lo[ok], hi[ok], dz[ok], dp[ok]
        f = (a_z * dz) + (a_phi * dp)                  # Eq. 2: two rounded products, one rounded sum
        # directed candidates R -> S in both directions; per R the minimal f,
        # ties to the larger S
        cr = np.concatenate([lo, hi])
        cs = np.concatenate([hi, lo])
        cf = np.concatenate([f, f])
        order = np.lexsort((-cs, cf, cr))
        cr, cs = cr[order], cs[order]
        first = np.ones(cr.size, bool)
        first[1:] = cr[1:] != cr[:-1]
        partner = np.full(n, -1, np.int64)
        partner[cr[first]] = cs[first]
        # mutual choices merge into the larger ID
        r = cr[first]
        s = partner[r]
        mutual = (partner[s] == r) & (r < s)
        loser, winner = r[mutual], s[mutual]
        sum_z[winner] = sum_z[winner] + sum_z[loser]
        sum_p[winner] = sum_p[winner] + sum_p[loser]
        size[winner] += size[loser]
        size[loser] = 0
        mean_z[winner] = sum_z[winner] / size[winner].astype(np.float32)
        mean_p[winner] = sum_p[winner] / size[winner].astype(np.float32)
        parent = np.arange(n, dtype=np.int64)
        parent[loser] = winner
        label = parent[label]
        rounds += 1
        counts.append(int(np.count_nonzero(size)))
    return (label.reshape(h, w).astype(np.int32), rounds, counts, mean_z, mean_p, size)


def brute(z, d, intensity, t_z=T_Z, t_phi=T_PHI, alpha_z=ALPHA_Z, alpha_phi=ALPHA_PHI):
    """The same rounds written loop by loop over explicit pixel sets (tiny
    grids only): regions as dicts {id: set of pixels}, neighbours found by
    scanning each member pixel's four neighbours.  Returns (labels, rounds)."""
    z = _f32(z)
    h, w = z.shape
    t_z, t_phi, a_z, a_phi = (np.float32(v) for v in (t_z, t_phi, alpha_z, alpha_phi))
    ph = phi(d, intensity)
    members = {y * w + x: {(y, x)} for y in range(h) for x in range(w)}
    sz = {k: np.float32(z[k // w, k % w]) for k in members}
    sp = {k: np.float32(ph[k // w, k % w]) for k in members}
    mz, mp = dict(sz), dict(sp)
    owner = {(y, x): y * w + x for y in range(h) for x in range(w)}
    rounds = 0
    while True:
        choice = {}
        for R, pix in members.items():
            best = None
            for (y, x) in pix:
                for (yy, xx) in ((y - 1, x), (y + 1, x), (y, x - 1), (y, x + 1)):
                    if not (0 <= yy < h and 0 <= xx < w):
                        continue
                    S = owner[(yy, xx)]
                    if S == R:
                        continue
                    dz = np.float32(abs(np.float32(mz[R] - mz[S])))
                    dp = np.float32(abs(np.float32(mp[R] - mp[S])))
                    if dz > t_z or dp > t_phi:
                        continue
                    f = np.float32(np.float32(a_z * dz) + np.float32(a_phi * dp))
                    if best is None or f < best[0] or (f == best[0] and S > best[1]):
                        best = (f, S)
            if best is not None:
                choice[R] = best[1]
        if not choice:
            break
        for R in sorted(choice):
            S = choice[R]
            if R < S and choice.get(S) == R:
                members[S] |= members.pop(R)
                for p in members[S]:
                    owner[p] = S
                sz[S] = np.float32(sz[S] + sz[R])
                sp[S] = np.float32(sp[S] + sp[R])
                cnt = np.float32(len(members[S]))
                mz[S] = np.float32(sz[S] / cnt)
                mp[S] = np.float32(sp[S] / cnt)
        rounds += 1
    labels = np.empty((h, w), np.int32)
    for (y, x), k in owner.items():
        labels[y, x] = k
    return labels, rounds
