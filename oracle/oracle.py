"""ctypes front end of the CPU oracle (nqs_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py. The CUDA library never imports or links this.
Each function restates a step of the method in FP64 (see nqs_oracle.h for the
conventions and the paper passages).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "nqs_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "nqs_oracle.h"))):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class Ham(C.Structure):
    _fields_ = [("K", C.c_int), ("n_alpha", C.c_int), ("n_beta", C.c_int),
                ("h1e", C.c_void_p), ("eri", C.c_void_p), ("e_core", C.c_double)]


class Ansatz(C.Structure):
    _fields_ = [("K", C.c_int), ("D", C.c_int), ("n_edges", C.c_int),
                ("pred_ptr", C.c_void_p), ("pred_idx", C.c_void_p), ("tensors", C.c_void_p),
                ("n_hidden", C.c_int), ("rbm_W", C.c_void_p), ("rbm_b", C.c_void_p),
                ("readout", C.c_int), ("n_alpha", C.c_int), ("n_beta", C.c_int),
                ("rnn_v", C.c_void_p), ("rnn_eta", C.c_void_p), ("rnn_w", C.c_void_p),
                ("rnn_c", C.c_void_p), ("corr", C.c_int), ("rbm_W2", C.c_void_p),
                ("tucker_rank", C.c_void_p), ("tucker", C.c_void_p)]


class SampleOut(C.Structure):
    _fields_ = [("e_loc", C.c_double), ("e_det", C.c_double), ("e_stoch", C.c_double),
                ("h_diag", C.c_double), ("e_abs", C.c_double), ("e_cond", C.c_double),
                ("log_abs_psi", C.c_double),
                ("log_f", C.c_double),
                ("sign_psi", C.c_int), ("n_det", C.c_int64), ("n_rem", C.c_int64),
                ("w_total", C.c_uint64), ("w_shift", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.or_n_conn.restype = C.c_int64
            _lib.or_diag.restype = C.c_double
            _lib.or_log_psi_p1.restype = C.c_double
            _lib.or_connected.restype = C.c_int64
    return _lib


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


class Problem:
    """Holds contiguous copies of a workloads.System (plus its ERI) so that the
    pointers handed to C stay alive."""

    def __init__(self, sys, eri=None):
        self.sys = sys
        self.h1e = _c(sys.h1e, np.float64)
        self.eri = _c(eri if eri is not None else build_eri(sys.chol), np.float64)
        self.tensors = _c(sys.tensors, np.float64)
        self.pred_ptr = _c(sys.pred_ptr, np.int32)
        self.pred_idx = _c(sys.pred_idx, np.int32)
        self.W = _c(sys.rbm_W, np.float64)
        self.b = _c(sys.rbm_b, np.float64)
        self.ham = Ham(sys.K, sys.n_alpha, sys.n_beta, self.h1e.ctypes.data,
                       self.eri.ctypes.data, float(sys.e_core))
        rnn = getattr(sys, "rnn", None)          # (v, eta, w, c) of the normalised readout
        self.rnn = None if rnn is None else tuple(_c(x, np.float64) for x in rnn)
        self.W2 = _c(getattr(sys, "rbm_W2", None), np.float64)
        tk = getattr(sys, "tucker", None)        # (ranks [K], packed parameters) of the tensor term
        self.tk_rank = None if tk is None else _c(tk[0], np.int32)
        self.tk = None if tk is None else _c(tk[1], np.float64)
        ptr = lambda a: a.ctypes.data if a is not None else None
        self.ans = Ansatz(sys.K, sys.D, int(self.tensors.shape[0]),
                          ptr(self.pred_ptr), ptr(self.pred_idx),
                          self.tensors.ctypes.data, sys.n_hidden, ptr(self.W), ptr(self.b),
                          1 if self.rnn is not None else 0, sys.n_alpha, sys.n_beta,
                          *(ptr(x) for x in (self.rnn or (None,) * 4)),
                          int(getattr(sys, "corr", 0)), ptr(self.W2), ptr(self.tk_rank), ptr(self.tk))


def build_eri(chol):
    """(pq|rs) = sum_x L^x_pq L^x_rs, ascending x with fma (Eq. Ham integrals)."""
    L = _c(chol, np.float64)
    nchol, K, _ = L.shape
    eri = np.empty(K ** 4, np.float64)
    lib().or_build_eri(K, nchol, _p(L), _p(eri))
    return eri


def n_conn(K, na, nb):
    return int(lib().or_n_conn(K, na, nb))


def diag(P: Problem, det):
    d = _c(det, np.uint64)
    return float(lib().or_diag(C.byref(P.ham), _p(d)))


def connected(P: Problem, det):
    """All singles and doubles of ``det`` in canonical order: (dets, H, sign)."""
    d = _c(det, np.uint64)
    nc = n_conn(P.sys.K, P.sys.n_alpha, P.sys.n_beta)
    dets = np.empty((nc, 2), np.uint64)
    H = np.empty(nc, np.float64)
    sg = np.empty(nc, np.int8)
    got = lib().or_connected(C.byref(P.ham), _p(d), _p(dets), _p(H), _p(sg))
    assert got == nc
    return dets, H, sg


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, np.uint64)
    lib().or_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def log_psi(P: Problem, det):
    """(log|psi|, sign, log f) with the full K-site product."""
    d = _c(det, np.uint64)
    la = C.c_double()
    sg = C.c_int()
    lf = C.c_double()
    lib().or_log_psi(C.byref(P.ans), _p(d), C.byref(la), C.byref(sg), C.byref(lf))
    return la.value, sg.value, lf.value


def log_psi_p1(P: Problem, det):
    """log P1: first-order rounding bound of the tensor-network contraction."""
    d = _c(det, np.uint64)
    return float(lib().or_log_psi_p1(C.byref(P.ans), _p(d)))


def draws(P: Problem, det, sample_index, eps, n_draws, seed):
    d = _c(det, np.uint64)
    ranks = np.empty(max(n_draws, 1), np.int64)
    W = C.c_uint64()
    sh = C.c_int()
    lib().or_draws(C.byref(P.ham), _p(d), C.c_int64(sample_index), C.c_double(eps),
                   n_draws, C.c_uint64(seed), _p(ranks), C.byref(W), C.byref(sh))
    return ranks[:n_draws], int(W.value), int(sh.value)


SAMPLE_DTYPE = np.dtype([("e_loc", "f8"), ("e_det", "f8"), ("e_stoch", "f8"),
                         ("h_diag", "f8"), ("e_abs", "f8"), ("e_cond", "f8"), ("log_abs_psi", "f8"),
                         ("log_f", "f8"),
                         ("sign_psi", "i4"), ("n_det", "i8"), ("n_rem", "i8"),
                         ("w_total", "u8"), ("w_shift", "i4")], align=True)
assert SAMPLE_DTYPE.itemsize == C.sizeof(SampleOut)


def local_energy(P: Problem, samples=None, eps=None, n_draws=None, seed=None, threads=0, index=None,
                 cond=False):
    """Semistochastic E_loc for each sample (structured array, SAMPLE_DTYPE).
    ``index`` gives each sample's position in the batch (Philox counter);
    ``cond`` also fills e_cond (doubles the amplitude work)."""
    s = _c(P.sys.samples if samples is None else samples, np.uint64).reshape(-1, 2)
    idx = None if index is None else _c(index, np.int64)
    eps = P.sys.eps if eps is None else eps
    n_draws = P.sys.n_draws if n_draws is None else n_draws
    seed = P.sys.seed if seed is None else seed
    out = np.zeros(len(s), SAMPLE_DTYPE)
    lib().or_local_energy(C.byref(P.ham), C.byref(P.ans), _p(s), C.c_int64(len(s)),
                          C.c_double(eps), int(n_draws), C.c_uint64(seed), _p(out),
                          int(threads), _p(idx), int(bool(cond)))
    return out


def rnn_conditionals(P: Problem, det):
    """P~_i(s) of the normalised readout along ``det``, [K][4] (Sec. 2.2)."""
    d = _c(det, np.uint64)
    out = np.zeros((P.sys.K, 4), np.float64)
    lib().or_rnn_conditionals(C.byref(P.ans), _p(d), _p(out))
    return out


def sample(P: Problem, n_samples, seed, capacity=None):
    """Autoregressive sampling from |Phi|^2 (Sec. 2.1, Sec. 3): unique
    determinants [n][2] and their counts, in prefix order."""
    cap = int(n_samples if capacity is None else capacity)
    dets = np.zeros((max(cap, 1), 2), np.uint64)
    counts = np.zeros(max(cap, 1), np.float64)
    lib().or_sample.restype = C.c_int64
    n = lib().or_sample(C.byref(P.ans), C.c_int64(n_samples), C.c_uint64(seed), _p(dets), _p(counts),
                        C.c_int64(cap))
    n = int(n)
    return dets[:min(n, cap)], counts[:min(n, cap)], n


def grad_corr_W2(P: Problem, det):
    """d log|f| / d W2 of the Ising-RBM correlator, [N_h][2K][2K]."""
    d = _c(det, np.uint64)
    N = 2 * P.sys.K
    g = np.zeros((P.sys.n_hidden, N, N), np.float64)
    lib().or_grad_corr_W2(C.byref(P.ans), _p(d), _p(g))
    return g


def grad_log_psi(P: Problem, det):
    d = _c(det, np.uint64)
    sys = P.sys
    gt = np.zeros_like(P.tensors)
    gW = np.zeros_like(P.W) if P.W is not None else None
    gb = np.zeros_like(P.b) if P.b is not None else None
    lib().or_grad_log_psi(C.byref(P.ans), _p(d), _p(gt), _p(gW), _p(gb))
    return gt, gW, gb


def summary(out, counts, ):
    """Weighted energy, B and the reweighted local energy (Sec. 2.3), real f."""
    c = np.asarray(counts, np.float64)
    e = out["e_loc"]
    ebar = float(np.sum(c * e) / np.sum(c))
    lf = out["log_f"]
    m = np.max(2 * lf)
    B_scaled = float(np.sum(c * np.exp(2 * lf - m)) / np.sum(c))   # B / e^m
    e_tilde = np.exp(2 * lf - m) / B_scaled * e
    return ebar, B_scaled, m, e_tilde
