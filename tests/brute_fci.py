"""Brute-force second-quantised Hamiltonian for tiny systems (numpy).

Independent of the oracle: it builds <x'|H|x> by applying every term of
Eq. (Ham), H = sum_pq h_pq a+_p a_q + 1/4 sum_pqrs <pq||rs> a+_p a+_q a_s a_r,
to integer bitstrings over the 2K interleaved spin orbitals (bit s = 2p+spin),
with the phase of each operator taken as (-1)^(occupied bits below s). It
uses no Slater-Condon rule and no excitation enumeration.
"""
import numpy as np


def interleave(dets, K):
    """[alpha word, beta word] -> one integer with bit 2p+spin."""
    out = np.zeros(len(dets), dtype=np.int64)
    for p in range(K):
        out |= ((dets[:, 0].astype(np.int64) >> p) & 1) << (2 * p)
        out |= ((dets[:, 1].astype(np.int64) >> p) & 1) << (2 * p + 1)
    return out


def _popcount(x):
    x = x.copy()
    c = np.zeros_like(x)
    while np.any(x):
        c += x & 1
        x >>= 1
    return c


def _apply(x, valid, coef, s, create):
    """Apply a_s (create=False) or a+_s to the states x (vectorised)."""
    bit = (x >> s) & 1
    ok = valid & ((bit == 0) if create else (bit == 1))
    below = x & ((1 << s) - 1)
    ph = 1 - 2 * (_popcount(below) & 1)
    return x ^ (1 << s), ok, coef * ph


def spin_integrals(h1e, eri, K):
    """h_{pq} and <pq||rs> over spin orbitals (index 2p+spin)."""
    n = 2 * K
    sp = np.arange(n) % 2
    orb = np.arange(n) // 2
    hs = h1e[orb[:, None], orb[None, :]] * (sp[:, None] == sp[None, :])
    e4 = eri.reshape(K, K, K, K)
    # <pq|rs> = (pr|qs) d(sp,sr) d(sq,ss)
    P, Q, R, S = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), np.arange(n),
                             indexing="ij")
    phys = e4[orb[P], orb[R], orb[Q], orb[S]] * (sp[P] == sp[R]) * (sp[Q] == sp[S])
    anti = phys - np.transpose(phys, (0, 1, 3, 2))
    return hs, anti


def hamiltonian(h1e, eri, K, dets, e_core=0.0):
    """Dense <x'|H|x> over the given determinant list (same order)."""
    x = interleave(np.asarray(dets, dtype=np.uint64), K)
    order = np.argsort(x)
    xs = x[order]
    N = len(x)
    H = np.zeros((N, N))
    hs, anti = spin_integrals(h1e, eri, K)
    n = 2 * K
    ones = np.ones(N, dtype=np.int64)
    allv = np.ones(N, dtype=bool)

    def scatter(y, ok, coef, val):
        if not np.any(ok):
            return
        y, coef, col = y[ok], coef[ok], np.nonzero(ok)[0]
        pos = np.searchsorted(xs, y)
        good = (pos < N) & (xs[np.minimum(pos, N - 1)] == y)
        np.add.at(H, (order[pos[good]], col[good]), val * coef[good])

    for p in range(n):
        for q in range(n):
            if hs[p, q] == 0.0:
                continue
            y, ok, c = _apply(x, allv, ones, q, False)
            y, ok, c = _apply(y, ok, c, p, True)
            scatter(y, ok, c, hs[p, q])
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for s in range(n):
                    v = anti[p, q, r, s]
                    if v == 0.0:
                        continue
                    y, ok, c = _apply(x, allv, ones, r, False)
                    y, ok, c = _apply(y, ok, c, s, False)
                    y, ok, c = _apply(y, ok, c, q, True)
                    y, ok, c = _apply(y, ok, c, p, True)
                    scatter(y, ok, c, 0.25 * v)
    H += e_core * np.eye(N)
    return H
