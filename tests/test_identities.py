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
* The per-site correlator table: an object's factors from the tanh and
  cosh - 1 of its one or two site changes by the addition formulas, in FP64
  and in FP32 where the kernel uses them (denominator >= 1/2).
* Double-FP32 dot products (psi(n) of the mixed form, the re-evaluation's
  tables) within D 2^-46 of sum |m x|.
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


def _site_factors(d):
    """tanh d and cosh d - 1 (the per-site table entries), FP64."""
    return np.tanh(d), 2.0 * np.sinh(d / 2) ** 2


@pytest.mark.parametrize("seed", [4, 5])
def test_site_table_addition_formulas(seed):
    """The per-site correlator table (Eq. RBM): an object's factors from the
    tanh u and cosh - 1 c of its one or two site changes d1, d2:
      den = 1 + p + t s, s = u1 + u2, p = u1 u2, t = tanh theta,
      tanh(theta + d1 + d2) = (t + s + t p) / den,
      cosh(theta + d1 + d2) / cosh(theta) - 1 = (1 + e) den - 1,
      tanh(d1 + d2) = s / (1 + p),  cosh(d1 + d2) - 1 = (1 + e)(1 + p) - 1,
    with e = (1 + c1)(1 + c2) - 1 (d2 = 0 gives the one-site forms)."""
    rng = np.random.default_rng(seed)
    n = 20000
    theta = rng.normal(0, 1.5, n)
    for scale in (0.01, 0.3, 1.5):
        d1 = rng.normal(0, scale, n)
        d2 = np.where(rng.random(n) < 0.3, 0.0, rng.normal(0, scale, n))
        (u1, c1), (u2, c2) = _site_factors(d1), _site_factors(d2)
        t = np.tanh(theta)
        s, p = u1 + u2, u1 * u2
        e = c1 + c2 + c1 * c2
        den = 1 + p + t * s
        assert np.all(den > 0)
        d = d1 + d2
        # rounding grows as 1 / den (the cancellation the kernel's den >= 1/2 test avoids)
        err = np.abs((t + s + t * p) / den - np.tanh(theta + d))
        assert np.all(err <= 1e-14 / den)
        assert np.max(err[den >= 0.5]) <= 16 * 2.0 ** -53
        ref_pl = np.expm1(np.log(np.cosh(theta + d)) - np.log(np.cosh(theta)))
        g = t * s + p                         # den - 1 formed directly, as the kernel does
        np.testing.assert_allclose(e + g + e * g, ref_pl, rtol=1e-10, atol=1e-13)
        np.testing.assert_allclose(s / (1 + p), np.tanh(d), rtol=0, atol=1e-13)
        # formed as e + p + e p (the kernel's order); when opposite changes cancel
        # the error is absolute, relative to the factor PR itself (~1)
        np.testing.assert_allclose(e + p + e * p, 2.0 * np.sinh(d / 2) ** 2, rtol=1e-10, atol=1e-13)


def test_site_table_formulas_in_float32_above_the_threshold():
    """The FP32 kernel evaluates the left factors from FP32-rounded table
    entries only when den >= 1/2 (else directly from theta + d): there the
    tanh and P - 1 terms stay within a few FP32 units of the FP64 values."""
    f = np.float32
    rng = np.random.default_rng(9)
    n = 50000
    theta = rng.normal(0, 1.5, n)
    d1, d2 = rng.normal(0, 0.3, n), rng.normal(0, 0.3, n)
    (u1, c1), (u2, c2) = _site_factors(d1), _site_factors(d2)
    t = np.tanh(theta).astype(f)
    u1, c1, u2, c2 = (x.astype(f) for x in (u1, c1, u2, c2))
    s, p = u1 + u2, u1 * u2
    e = c1 + c2 + c1 * c2
    den = t * s + (f(1) + p)
    keep = den >= f(0.5)
    assert keep.mean() > 0.95
    val = (t * p + (t + s)) / den
    g = t * s + p
    y = e * g + (e + g)
    d = d1 + d2
    ref_t = np.tanh(theta + d)
    ref_y = np.expm1(np.log(np.cosh(theta + d)) - np.log(np.cosh(theta)))
    assert np.max(np.abs(val[keep] - ref_t[keep])) < 16 * 2.0 ** -24
    assert np.max(np.abs(y[keep] - ref_y[keep]) / (1 + np.abs(ref_y[keep]))) < 16 * 2.0 ** -24


def _fmaf(a, b, c):
    """float32 fused multiply-add (the product of two floats is exact in FP64)."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def test_double_float_dot_products():
    """psi(n) of the mixed form and the re-evaluation's tables use double-FP32
    dot products: matrix and vector as (hi, lo) float pairs, each term the
    error-free product by FMA plus the cross terms, summed with Knuth's
    two-sum into an unnormalised pair. Emulated here in float32 with the
    kernels' operation order: the result is within D 2^-46 of sum |m x| of
    the exact FP64 dot product."""
    f = np.float32
    rng = np.random.default_rng(11)
    for D in (32, 64, 256):
        for _ in range(20):
            m = rng.normal(0, 1, D)
            x = rng.normal(0, 1, D) * np.exp(rng.normal(0, 2, D))
            mh = m.astype(f); ml = (m - mh.astype(np.float64)).astype(f)
            xh = x.astype(f); xl = (x - xh.astype(np.float64)).astype(f)
            hi, lo = f(0), f(0)
            for k in range(D):
                pr = f(mh[k] * xh[k])
                pe = f(_fmaf(mh[k], xh[k], -pr) + _fmaf(mh[k], xl[k], f(ml[k] * xh[k])))
                u = f(hi + pr)
                z = f(u - hi)
                lo = f(lo + f(f(f(hi - f(u - z)) + f(pr - z)) + pe))
                hi = u
            got = float(hi) + float(lo)
            exact = math.fsum(float(a) * float(b) for a, b in zip(m, x))
            scale = math.fsum(abs(float(a) * float(b)) for a, b in zip(m, x))
            assert abs(got - exact) <= D * 2.0 ** -46 * scale
