"""Test-side helpers: the dense matrix represented by the exported layer layout of
include/hsweep.h, and random layers in that layout.  No method arithmetic beyond
assembling the blocks the layout documents."""
import numpy as np


def tree(n, leaf=8):
    L = 0
    while -(-n // (1 << L)) > leaf:
        L += 1
    nn = 1 << (L + 1)
    lo, sz = [0] * nn, [0] * nn
    sz[1] = n
    for v in range(1, nn // 2):
        a = (sz[v] + 1) // 2
        lo[2 * v], sz[2 * v] = lo[v], a
        lo[2 * v + 1], sz[2 * v + 1] = lo[v] + a, sz[v] - a
    return L, lo, sz


def layer_to_dense(n, leaf, r_max, leaves, fac, ranks):
    """Dense T from the host layer layout (leaves column-major, F_v column-major)."""
    L, lo, sz = tree(n, leaf)
    T = np.zeros((n, n), complex)
    for lam in range(1 << L, 1 << (L + 1)):
        k = lam - (1 << L)
        D = leaves[k * leaf * leaf:(k + 1) * leaf * leaf].reshape(leaf, leaf).T
        s = sz[lam]
        T[lo[lam]:lo[lam] + s, lo[lam]:lo[lam] + s] = D[:s, :s]
    F = {}
    o = 0
    for v in range(2, 1 << (L + 1)):
        F[v] = fac[o:o + sz[v] * r_max].reshape(r_max, sz[v]).T[:, :ranks[v]]
        o += sz[v] * r_max
    for t in range(1, 1 << L):
        a, b = 2 * t, 2 * t + 1
        blk = F[a] @ F[b].T
        T[lo[a]:lo[a] + sz[a], lo[b]:lo[b] + sz[b]] = blk
        T[lo[b]:lo[b] + sz[b], lo[a]:lo[a] + sz[a]] = blk.T
    return T


def random_layer(n, leaf, r_max, rng, scale, full_rank_pairs=False):
    """A random symmetric-storage layer: leaves, factors and ranks (siblings equal)."""
    L, lo, sz = tree(n, leaf)
    nleaves = 1 << L
    leaves = np.zeros(nleaves * leaf * leaf, complex)
    for k in range(nleaves):
        s = sz[nleaves + k]
        D = np.zeros((leaf, leaf), complex)
        D[:s, :s] = scale * (rng.standard_normal((s, s)) + 1j * rng.standard_normal((s, s)))
        leaves[k * leaf * leaf:(k + 1) * leaf * leaf] = D.T.ravel()
    ranks = np.zeros(1 << (L + 1), np.int32)
    for t in range(1, 1 << L):
        cap = min(r_max, sz[2 * t], sz[2 * t + 1])
        r = cap if full_rank_pairs else int(rng.integers(0, cap + 1))
        ranks[2 * t] = ranks[2 * t + 1] = r
    parts = []
    for v in range(2, 1 << (L + 1)):
        Fm = np.zeros((sz[v], r_max), complex)
        r = ranks[v]
        Fm[:, :r] = np.sqrt(scale / max(1, r)) * (rng.standard_normal((sz[v], r)) + 1j * rng.standard_normal((sz[v], r)))
        parts.append(Fm.T.ravel())
    return leaves, np.concatenate(parts), ranks


def strong_to_dense(n, leaf, R, rec, recoff, rstride):
    """Dense T from the strongly admissible records of hsweep_strong_export: per row the
    blocks of its leaf and the neighbouring leaves, and the rows of W_{v,t}; every
    well-separated pair (u, w) is W_{u,t(w)} W_{w,t(u)}^t."""
    L, lo, sz = tree(n, leaf)
    nleaves = 1 << L

    def il(c):
        return (-3, -2, 2) if c & 1 else (-2, 2, 3)

    T = np.zeros((n, n), complex)
    W = {}
    for j in range(nleaves):
        lam = nleaves + j
        s = sz[lam]
        sl = sz[lam - 1] if j > 0 else 0
        sr = sz[lam + 1] if j < nleaves - 1 else 0
        wb = s + sl + sr
        for i in range(s):
            base = int(recoff[j]) + i * int(rstride[j])
            row = rec[base:base + wb + 3 * R * (L - 1)]
            g = lo[lam] + i
            T[g, lo[lam]:lo[lam] + s] += row[:s]
            if sl:
                T[g, lo[lam - 1]:lo[lam - 1] + sl] += row[s:s + sl]
            if sr:
                T[g, lo[lam + 1]:lo[lam + 1] + sr] += row[s + sl:wb]
            for d in range(2, L + 1):
                v = lam >> (L - d)
                iv = lo[lam] + i - lo[v]
                for t in range(3):
                    o = wb + (d - 2) * 3 * R + t * R
                    W.setdefault((v, t), np.zeros((sz[v], R), complex))[iv] = row[o:o + R]
    for (v, t), Wv in W.items():
        d = v.bit_length() - 1
        vl = v - (1 << d)
        pl = vl + il(vl)[t]
        if not 0 <= pl < (1 << d):
            assert not Wv.any()
            continue
        p = (1 << d) + pl
        tp = il(pl).index(-il(vl)[t])
        T[lo[v]:lo[v] + sz[v], lo[p]:lo[p] + sz[p]] += Wv @ W[(p, tp)].T
    return T
