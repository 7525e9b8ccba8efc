"""Pins of the oracle's Hamiltonian: Slater-Condon elements, signs, the
canonical enumeration and the integral build (Eq. Ham, Sec. 2.1 and 2.4).

Each pin is independent of the oracle's own code: a brute-force
second-quantised Hamiltonian, closed forms, symmetries, and counting.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_19276_gb300 import workloads as W
from tests import brute_fci


def dense_oracle_H(P, dets):
    """Dense <m|H|n> assembled from the oracle's diagonal and connected lists."""
    key = {(int(a), int(b)): i for i, (a, b) in enumerate(dets)}
    N = len(dets)
    H = np.zeros((N, N))
    for j, d in enumerate(dets):
        H[j, j] = O.diag(P, d)
        md, hv, _ = O.connected(P, d)
        for m, v in zip(md, hv):
            H[key[(int(m[0]), int(m[1]))], j] += v
    return H


def test_eri_matches_einsum_and_is_eightfold_symmetric():
    sys_ = W.small_chain()
    eri = O.build_eri(sys_.chol).reshape((sys_.K,) * 4)
    ref = np.einsum("xpq,xrs->pqrs", sys_.chol, sys_.chol)
    assert np.max(np.abs(eri - ref)) < 1e-14
    # exact (bitwise) 8-fold symmetry: needed for H_nm = H_mn bitwise
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.array_equal(eri, np.transpose(eri, perm))


@pytest.mark.parametrize("K,na,nb", [(4, 2, 2), (5, 3, 2), (6, 3, 3), (8, 4, 4), (7, 1, 5)])
def test_n_conn_counts_every_single_and_double(K, na, nb):
    dets = W.all_dets(K, na, nb)
    x = brute_fci.interleave(dets, K)
    # independent count: determinants at excitation level 1 or 2 from dets[0]
    diff = np.array([bin(int(v) ^ int(x[0])).count("1") for v in x])
    assert np.sum((diff == 2) | (diff == 4)) == O.n_conn(K, na, nb)


@pytest.mark.parametrize("K,na,nb,seed", [(4, 2, 2, 1), (4, 1, 2, 2), (5, 3, 2, 3),
                                          (5, 2, 2, 4), (6, 3, 3, 5)])
def test_oracle_H_equals_brute_force_second_quantisation(K, na, nb, seed):
    sys_ = W.tiny_system(K=K, na=na, nb=nb, seed=seed)
    P = O.Problem(sys_)
    dets = W.all_dets(K, na, nb)
    Hb = brute_fci.hamiltonian(sys_.h1e, P.eri, K, dets)
    Ho = dense_oracle_H(P, dets)
    assert np.max(np.abs(Hb - Ho)) < 1e-13
    # the connected lists cover every nonzero off-diagonal element
    off = np.abs(Hb) > 1e-12
    np.fill_diagonal(off, False)
    assert np.all(Ho[off] != 0.0)


def test_hermitian_bitwise_on_small_chain():
    sys_ = W.small_chain()
    P = O.Problem(sys_)
    for d in sys_.samples[:16]:
        md, hv, _ = O.connected(P, d)
        for m, v in zip(md[::7], hv[::7]):
            back_d, back_h, _ = O.connected(P, m)
            hit = np.nonzero((back_d[:, 0] == d[0]) & (back_d[:, 1] == d[1]))[0]
            assert len(hit) == 1
            assert back_h[hit[0]] == v  # bitwise


def test_one_body_closed_form():
    """With (pq|rs)=0 the ground energy is the sum of the lowest N_a and N_b
    orbital energies of h (a textbook closed form)."""
    K, na, nb = 6, 3, 2
    sys_ = W.tiny_system(K=K, na=na, nb=nb, seed=11)
    P = O.Problem(sys_, eri=np.zeros(K ** 4))
    dets = W.all_dets(K, na, nb)
    Ho = dense_oracle_H(P, dets)
    e0 = np.linalg.eigvalsh(Ho)[0]
    eps = np.linalg.eigvalsh(sys_.h1e)
    assert abs(e0 - (eps[:na].sum() + eps[:nb].sum())) < 1e-12


def test_canonical_order_blocks():
    """Ranks run over [S_a, S_b, D_aa, D_bb, D_ab] with positions among the
    occupied / empty orbitals ascending and pairs lexicographic."""
    K, na, nb = 5, 2, 2
    sys_ = W.tiny_system(K=K, na=na, nb=nb, seed=3)
    P = O.Problem(sys_)
    n = np.array([0b00101, 0b10010], np.uint64)
    md, _, _ = O.connected(P, n)
    occ = [[0, 2], [1, 4]]
    vir = [[1, 3, 4], [0, 2, 3]]
    exp = []
    for sp in range(2):
        for i in occ[sp]:
            for a in vir[sp]:
                m = n.copy(); m[sp] ^= np.uint64((1 << i) | (1 << a)); exp.append(m)
    for sp in range(2):
        for i, j in itertools.combinations(occ[sp], 2):
            for a, b in itertools.combinations(vir[sp], 2):
                m = n.copy(); m[sp] ^= np.uint64((1 << i) | (1 << j) | (1 << a) | (1 << b))
                exp.append(m)
    for i in occ[0]:
        for a in vir[0]:
            for j in occ[1]:
                for b in vir[1]:
                    m = n.copy(); m[0] ^= np.uint64((1 << i) | (1 << a))
                    m[1] ^= np.uint64((1 << j) | (1 << b)); exp.append(m)
    assert np.array_equal(md, np.array(exp, np.uint64))


def test_sixty_four_orbitals_use_the_top_bit():
    """K = 64 fills the 64-bit occupation words: a determinant with orbital 63
    occupied in both spins. Its connected list has n_conn entries that conserve
    both electron counts, every element is Hermitian bitwise, and every sign
    is the closed-form phase parity (Sec. 3 operator order)."""
    from tests.test_identities import _closed_parity, _interleave
    K, na, nb = 64, 2, 1
    sys_ = W.tiny_system(K=K, na=na, nb=nb, seed=13, chol_rank=6, n_samples=4)
    P = O.Problem(sys_)
    n = np.array([(1 << 63) | (1 << 20), 1 << 63], np.uint64)
    md, hv, sg = O.connected(P, n)
    c2 = lambda x: x * (x - 1) // 2
    assert len(md) == O.n_conn(K, na, nb) == (na * (K - na) + nb * (K - nb) + c2(na) * c2(K - na)
                                              + c2(nb) * c2(K - nb) + na * (K - na) * nb * (K - nb))
    pops = [bin(int(a)).count("1") for a in md[:, 0]], [bin(int(b)).count("1") for b in md[:, 1]]
    assert set(pops[0]) == {na} and set(pops[1]) == {nb}
    x = _interleave(n, K)
    top = 0
    for m, v, s in zip(md, hv, sg):
        y = _interleave(m, K)
        gone = [t for t in range(2 * K) if (x >> t & 1) and not (y >> t & 1)]
        new = [t for t in range(2 * K) if (y >> t & 1) and not (x >> t & 1)]
        top += (2 * 63) in gone or (2 * 63 + 1) in gone
        if len(gone) == 1:
            par = _closed_parity(x, gone[0], new[0])
        else:
            i, j = gone
            a, b = new if ((i & 1) == (j & 1) or (new[0] & 1) == (i & 1)) else new[::-1]
            par = _closed_parity(x, i, a, j, b)
        assert (-1) ** par == int(s)
    assert top > 0                       # excitations out of orbital 63 were enumerated
    for m, v in zip(md[::97], hv[::97]):
        back_d, back_h, _ = O.connected(P, m)
        hit = np.nonzero((back_d[:, 0] == n[0]) & (back_d[:, 1] == n[1]))[0]
        assert len(hit) == 1 and back_h[hit[0]] == v
