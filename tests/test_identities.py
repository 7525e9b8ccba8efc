"""Identities the CUDA kernels rely on, checked on the CPU against independent
definitions (the GPU parity tests then check the kernels themselves).

* Fermionic phase in closed form: the sign of <m| a+_a a+_b a_j a_i |n> (the
  operators applied in that order, each counting the occupied spin orbitals
  below it, Sec. 3) has parity cb(i) + cb(j) + cb(b) + cb(a) + [i<j] + [i<b]
  + [j<b] + [i<a] + [j<a] + [b<a], with cb() counted in n; a single has
  cb(i) + cb(a) + [i<a]. Checked against sequential operator application and
  against the oracle's signs of every connected determinant.
* Correlator split (Eq. RBM): prod_k cosh(theta + dL + dR) / cosh(theta)
  = PL * PR * prod_k (1 + tanh(theta + dL) tanh(dR)), with
  PL = prod cosh(theta + dL) / cosh(theta) and PR = prod cosh(dR).
* The product recursion X <- X + y + X y carries prod (1 + y) - 1 without
  cancellation near 1.
"""
import math
import random

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_19276_gb300 import workloads as W


def _cb(x, s):
    """Occupied spin orbitals below s in the interleaved bitstring x."""
    return bin(x & ((1 << s) - 1)).count("1")


def _sequential_parity(x, ops):
    """Apply annihilators/creators in order; parity of the collected counts."""
    c = 0
    for s in ops:
        c += _cb(x, s)
        x ^= 1 << s
    return c & 1, x


def _closed_parity(x, i, a, j=None, b=None):
    if j is None:
        return (_cb(x, i) + _cb(x, a) + (i < a)) & 1
    order = (i < j) + (i < b) + (j < b) + (i < a) + (j < a) + (b < a)
    return (_cb(x, i) + _cb(x, j) + _cb(x, b) + _cb(x, a) + order) & 1


def test_phase_closed_form_matches_sequential_application():
    rng = random.Random(20250719)
    for _ in range(20000):
        n = 2 * rng.randint(2, 64)
        x = rng.getrandbits(n)
        occ = [s for s in range(n) if x >> s & 1]
        vir = [s for s in range(n) if not x >> s & 1]
        if len(occ) < 2 or len(vir) < 2:
            continue
        if rng.random() < 0.3:
            i, a = rng.choice(occ), rng.choice(vir)
            ref, _ = _sequential_parity(x, [i, a])
            assert _closed_parity(x, i, a) == ref
        else:
            i, j = rng.sample(occ, 2)
            a, b = rng.sample(vir, 2)
            ref, _ = _sequential_parity(x, [i, j, b, a])
            assert _closed_parity(x, i, a, j, b) == ref


def _interleave(det, K):
    x = 0
    for p in range(K):
        x |= ((int(det[0]) >> p) & 1) << (2 * p)
        x |= ((int(det[1]) >> p) & 1) << (2 * p + 1)
    return x


def test_phase_closed_form_matches_oracle_signs():
    """Every connected determinant of a few samples: the spin orbitals that
    change give (i, j) emptied and (a, b) filled; the canonical operator
    order puts the lower emptied orbital first (i < j) and, for doubles of
    one spin, the lower filled one in b (R8: pairs lexicographic)."""
    sys_ = W.tiny_system(K=7, na=3, nb=2, D=4, n_hidden=3, seed=5)
    P = O.Problem(sys_)
    K = sys_.K
    for det in sys_.samples[:6]:
        x = _interleave(det, K)
        dets, _, sg = O.connected(P, det)
        for m, s in zip(dets, sg):
            y = _interleave(m, K)
            gone = [t for t in range(2 * K) if (x >> t & 1) and not (y >> t & 1)]
            new = [t for t in range(2 * K) if (y >> t & 1) and not (x >> t & 1)]
            if len(gone) == 1:
                par = _closed_parity(x, gone[0], new[0])
            else:
                i, j = gone
                if (i & 1) == (j & 1):          # same spin: a < b in the pair order
                    a, b = new
                else:                           # alpha-beta: a takes i's spin
                    a, b = (new if (new[0] & 1) == (i & 1) else new[::-1])
                par = _closed_parity(x, i, a, j, b)
            assert (-1) ** par == int(s), (det, m)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_correlator_split_identity(seed):
    rng = np.random.default_rng(seed)
    nh = 100
    theta = rng.normal(0, 2.0, nh)
    for scale in (0.01, 0.3, 2.0):
        dL = rng.normal(0, scale, nh)
        dR = rng.normal(0, scale, nh)
        ref = np.sum(np.log(np.cosh(theta + dL + dR)) - np.log(np.cosh(theta)))
        logPL = np.sum(np.log(np.cosh(theta + dL)) - np.log(np.cosh(theta)))
        logPR = np.sum(np.log(np.cosh(dR)))
        prod = np.sum(np.log1p(np.tanh(theta + dL) * np.tanh(dR)))
        assert abs((logPL + logPR + prod) - ref) <= 1e-12 * max(1.0, abs(ref))


def test_product_recursion_keeps_the_small_part():
    rng = np.random.default_rng(7)
    y = rng.normal(0, 1e-9, 200)
    X = 0.0
    for v in y:
        X = X * v + (X + v)
    ref = math.fsum(y) + sum(y[i] * y[j] for i in range(len(y)) for j in range(i + 1, len(y)))
    assert abs(X - ref) <= 1e-12 * abs(ref)
    # the same product formed as prod(1 + y) - 1 loses most of its digits
    naive = float(np.prod(1.0 + y) - 1.0)
    assert abs(naive - ref) > abs(X - ref)


def test_series_for_cosh_and_sinh_in_float32():
    """The truncated series the FP32 correlator factors use for |d| <= 1."""
    f = np.float32
    d = np.concatenate([np.linspace(-1, 1, 4001), np.geomspace(1e-8, 1, 200)]).astype(f)
    z = d * d
    c = [f(1 / 3628800), f(1 / 40320), f(1 / 720), f(1 / 24), f(0.5)]
    ch1 = z * ((((c[0] * z + c[1]) * z + c[2]) * z + c[3]) * z + c[4])
    s = [f(1 / 39916800), f(1 / 362880), f(1 / 5040), f(1 / 120), f(1 / 6)]
    sh = (d * z) * ((((s[0] * z + s[1]) * z + s[2]) * z + s[3]) * z + s[4]) + d
    D = d.astype(np.float64)
    ref_ch1 = 2.0 * np.sinh(D / 2) ** 2
    ref_sh = np.sinh(D)
    nz = D != 0
    assert np.max(np.abs(ch1[nz] - ref_ch1[nz]) / ref_ch1[nz]) < 4 * 2.0 ** -24
    assert np.max(np.abs(sh[nz] - ref_sh[nz]) / np.abs(ref_sh[nz])) < 4 * 2.0 ** -24
