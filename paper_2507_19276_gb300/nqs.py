"""Python binding of the C ABI in include/nqs.h (ctypes; marshalling only).

Every function of the C library has a same-named Python function here taking
a context handle; `Context` wraps them with tensor-friendly signatures. Arrays
may be torch tensors (CUDA or CPU) or numpy arrays; their data pointers are
passed through as they are, so CUDA tensors stay on the device and host
arrays are staged by the library. All computation happens in libnqs.so: if it
cannot be loaded, import fails loudly. There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

NQS_OK = 0
NQS_PREC_FP64 = 0
NQS_PREC_MIXED = 1
NQS_PREC_FP64_SHARED = 2
STATUS = {0: "NQS_OK", 1: "NQS_ERR_INVALID_ARG", 2: "NQS_ERR_STATE", 3: "NQS_ERR_OOM",
          4: "NQS_ERR_CUDA", 5: "NQS_ERR_TIMEOUT", 6: "NQS_ERR_UNSUPPORTED"}


class NQSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


NQS_CORR_COSH = 0
NQS_CORR_COS = 1
NQS_CORR_ISING = 2


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("timing", C.c_int),
                ("sample_index_base", C.c_int64), ("energy_tolerance", C.c_double),
                ("grad_chunk", C.c_int), ("audit_samples", C.c_int),
                ("tile_blocks_per_sm", C.c_int), ("table_mb", C.c_int),
                ("reserved", C.c_int * 6)]


N_STAGES = 9
STAGES = ["env", "count", "write", "draw", "amp_det", "amp_draw", "final", "other", "tables"]


class EnergySummary(C.Structure):
    _fields_ = [("e_mean", C.c_double), ("sum_counts", C.c_double), ("log_B", C.c_double),
                ("e_tilde_mean", C.c_double), ("n_conn", C.c_int64), ("n_det", C.c_int64),
                ("n_draw_unique", C.c_int64), ("n_amplitudes", C.c_int64),
                ("span_sites", C.c_int64), ("matvecs", C.c_int64), ("n_refined", C.c_int64),
                ("e_error_bound", C.c_double), ("n_audited", C.c_int64),
                ("audit_rel_error", C.c_double), ("error_factor", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchItem(C.Structure):
    _fields_ = [("samples", C.c_void_p), ("counts", C.c_void_p), ("n_samples", C.c_int64),
                ("det_threshold", C.c_double), ("n_draws", C.c_int), ("philox_seed", C.c_uint64),
                ("e_loc", C.c_void_p), ("summary", C.POINTER(EnergySummary)), ("status", C.c_int),
                ("reweighted", C.c_int), ("grad_sites", C.c_void_p), ("grad_W", C.c_void_p),
                ("grad_b", C.c_void_p)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libnqs.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = C.CDLL(path)
        vp, i64, dbl, u64 = C.c_void_p, C.c_int64, C.c_double, C.c_uint64
        sig = {
            "nqs_create": [C.POINTER(vp), C.c_int, vp],
            "nqs_destroy": [vp],
            "nqs_set_options": [vp, C.POINTER(Options)],
            "nqs_stage_times": [vp, vp, vp, C.c_int],
            "nqs_set_hamiltonian": [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, dbl],
            "nqs_set_ansatz": [vp, vp, C.c_int, C.c_int, vp, vp, vp, vp, C.c_int],
            "nqs_connected": [vp, vp, i64, dbl, vp, vp, vp, vp, vp, i64],
            "nqs_amplitude": [vp, vp, i64, vp, vp],
            "nqs_draws": [vp, vp, i64, dbl, C.c_int, u64, vp, vp],
            "nqs_draws_noalloc": [vp, vp, i64, dbl, C.c_int, u64, vp, vp],
            "nqs_local_energy": [vp, vp, vp, i64, dbl, C.c_int, u64, vp, C.POINTER(EnergySummary)],
            "nqs_grad_log_psi_vjp": [vp, vp, vp, i64, vp, vp, vp],
            "nqs_grad_log_psi_vjp2": [vp, vp, vp, i64, vp, vp, vp, vp],
            "nqs_energy_gradient": [vp, vp, vp, i64, dbl, C.c_int, u64, C.c_int, vp, vp, vp, vp, vp,
                                    C.POINTER(EnergySummary)],
            "nqs_local_energy_batch": [C.POINTER(vp), C.c_int, C.POINTER(BatchItem), C.c_int],
            "nqs_set_readout": [vp, vp, vp, vp, vp, C.c_int],
            "nqs_set_correlator": [vp, C.c_int, vp],
            "nqs_set_tensor_term": [vp, vp, vp, i64],
            "nqs_sample": [vp, i64, u64, vp, vp, i64, C.POINTER(i64)],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_int
        lib.nqs_last_error.argtypes = [vp]
        lib.nqs_last_error.restype = C.c_char_p
        _lib = lib
        return lib


def exported_symbols():
    return ["nqs_create", "nqs_destroy", "nqs_last_error", "nqs_set_options", "nqs_stage_times",
            "nqs_set_hamiltonian", "nqs_set_ansatz", "nqs_connected", "nqs_amplitude",
            "nqs_draws", "nqs_draws_noalloc", "nqs_local_energy", "nqs_local_energy_batch",
            "nqs_grad_log_psi_vjp", "nqs_grad_log_psi_vjp2", "nqs_energy_gradient", "nqs_set_readout",
            "nqs_set_correlator", "nqs_set_tensor_term", "nqs_sample"]


def _ptr(x):
    """Data pointer of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported array type {type(x)}")


def _check(ctx, status):
    if status != NQS_OK:
        msg = load().nqs_last_error(ctx)
        raise NQSError(status, (msg or b"").decode())


# ---- same-named wrappers of the C ABI --------------------------------------

def nqs_create(device: int = 0, stream: int = 0):
    h = C.c_void_p()
    st = load().nqs_create(C.byref(h), device, C.c_void_p(stream or None))
    if st != NQS_OK:
        raise NQSError(st, f"nqs_create(device={device}) failed")
    return h


def nqs_destroy(ctx):
    load().nqs_destroy(ctx)


def nqs_last_error(ctx) -> str:
    return (load().nqs_last_error(ctx) or b"").decode()


def nqs_set_options(ctx, precision: int, timing: int = 0, sample_index_base: int = 0,
                    energy_tolerance: float = 0.0, grad_chunk: int = 0, audit_samples: int = 0,
                    tile_blocks_per_sm: int = 0, table_mb: int = 0):
    o = Options()
    o.precision = precision
    o.timing = timing
    o.sample_index_base = sample_index_base
    o.energy_tolerance = energy_tolerance
    o.grad_chunk = grad_chunk
    o.audit_samples = audit_samples
    o.tile_blocks_per_sm = tile_blocks_per_sm
    o.table_mb = table_mb
    _check(ctx, load().nqs_set_options(ctx, C.byref(o)))


def nqs_set_readout(ctx, v, eta, w, c, constrained=1):
    _check(ctx, load().nqs_set_readout(ctx, _ptr(v), _ptr(eta), _ptr(w), _ptr(c), int(constrained)))


def nqs_set_correlator(ctx, kind, W2=None):
    _check(ctx, load().nqs_set_correlator(ctx, int(kind), _ptr(W2)))


def nqs_set_tensor_term(ctx, ranks, params, n_params):
    _check(ctx, load().nqs_set_tensor_term(ctx, _ptr(ranks), _ptr(params), int(n_params)))


def nqs_sample(ctx, n_samples, seed, samples, counts, capacity):
    """Returns the number of unique samples (also when capacity is too small,
    in which case NQSError is raised after the count is known)."""
    n = C.c_int64(0)
    st = load().nqs_sample(ctx, int(n_samples), int(seed), _ptr(samples), _ptr(counts), int(capacity),
                           C.byref(n))
    if st != NQS_OK:
        err = NQSError(st, nqs_last_error(ctx))
        err.n_unique = n.value
        raise err
    return n.value


def nqs_grad_log_psi_vjp2(ctx, samples, u, Ns, grad_sites, grad_W, grad_b, grad_W2):
    _check(ctx, load().nqs_grad_log_psi_vjp2(ctx, _ptr(samples), _ptr(u), Ns, _ptr(grad_sites),
                                             _ptr(grad_W), _ptr(grad_b), _ptr(grad_W2)))


def nqs_energy_gradient(ctx, samples, counts, Ns, eps, n_draws, seed, reweighted, grad_sites, grad_W,
                        grad_b, grad_W2, e_loc=None, summary=None):
    _check(ctx, load().nqs_energy_gradient(ctx, _ptr(samples), _ptr(counts), Ns, float(eps), n_draws, seed,
                                           int(reweighted), _ptr(grad_sites), _ptr(grad_W), _ptr(grad_b),
                                           _ptr(grad_W2), _ptr(e_loc),
                                           C.byref(summary) if summary is not None else None))


def nqs_stage_times(ctx, ms, launches, n=N_STAGES):
    _check(ctx, load().nqs_stage_times(ctx, _ptr(ms), _ptr(launches), n))


def nqs_set_hamiltonian(ctx, h1e, chol_or_eri, n_chol, n_orb, n_alpha, n_beta, e_core=0.0):
    _check(ctx, load().nqs_set_hamiltonian(ctx, _ptr(h1e), _ptr(chol_or_eri), n_chol, n_orb,
                                           n_alpha, n_beta, float(e_core)))


def nqs_set_ansatz(ctx, tensors, n_edges, bond_dim, pred_ptr, pred_idx, rbm_W, rbm_b, n_hidden):
    _check(ctx, load().nqs_set_ansatz(ctx, _ptr(tensors), n_edges, bond_dim, _ptr(pred_ptr),
                                      _ptr(pred_idx), _ptr(rbm_W), _ptr(rbm_b), n_hidden))


def nqs_connected(ctx, samples, Ns, eps, offsets, rank, dets, H, sign, capacity):
    _check(ctx, load().nqs_connected(ctx, _ptr(samples), Ns, float(eps), _ptr(offsets), _ptr(rank),
                                     _ptr(dets), _ptr(H), _ptr(sign), capacity))


def nqs_amplitude(ctx, dets, n, log_abs, sign):
    _check(ctx, load().nqs_amplitude(ctx, _ptr(dets), n, _ptr(log_abs), _ptr(sign)))


def nqs_draws(ctx, samples, Ns, eps, n_draws, seed, ranks, w_total):
    _check(ctx, load().nqs_draws(ctx, _ptr(samples), Ns, float(eps), n_draws, seed, _ptr(ranks),
                                 _ptr(w_total)))


def nqs_draws_noalloc(ctx, samples, Ns, eps, n_draws, seed, ranks, w_total):
    """nqs_draws using only the library's fixed scratch array (device pointers only)."""
    _check(ctx, load().nqs_draws_noalloc(ctx, _ptr(samples), Ns, float(eps), n_draws, seed,
                                         _ptr(ranks), _ptr(w_total)))


def nqs_local_energy(ctx, samples, counts, Ns, eps, n_draws, seed, e_loc, summary=None):
    _check(ctx, load().nqs_local_energy(ctx, _ptr(samples), _ptr(counts), Ns, float(eps), n_draws,
                                        seed, _ptr(e_loc),
                                        C.byref(summary) if summary is not None else None))


def nqs_local_energy_batch(ctxs, items, n_workers=0):
    """ctxs: context handles; items: a ctypes array of BatchItem (statuses are
    written back). Raises NQSError naming the first failing system."""
    n = len(ctxs)
    arr = (C.c_void_p * n)(*[C.c_void_p(h.value if isinstance(h, C.c_void_p) else h) for h in ctxs])
    st = load().nqs_local_energy_batch(arr, n, items, n_workers)
    if st != NQS_OK:
        bad = [i for i in range(n) if items[i].status != NQS_OK]
        if not bad:
            raise NQSError(st, "invalid batch (null or repeated context)")
        msg = load().nqs_last_error(ctxs[bad[0]])
        raise NQSError(items[bad[0]].status, f"system {bad[0]}: " + (msg or b"").decode())


def nqs_grad_log_psi_vjp(ctx, samples, u, Ns, grad_sites, grad_W, grad_b):
    _check(ctx, load().nqs_grad_log_psi_vjp(ctx, _ptr(samples), _ptr(u), Ns, _ptr(grad_sites),
                                            _ptr(grad_W), _ptr(grad_b)))


# ---- convenience wrapper ----------------------------------------------------

def _np(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


class Context:
    """One library context bound to a device and a CUDA stream."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self.device = device
        self.h = nqs_create(device, stream)
        self.K = None
        self.n_edges = None
        self.D = None
        self.n_hidden = 0

    def close(self):
        if self.h is not None:
            nqs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision: int, timing: bool = False, sample_index_base: int = 0,
                      energy_tolerance: float = 0.0, grad_chunk: int = 0, audit_samples: int = 0,
                      tile_blocks_per_sm: int = 0, table_mb: int = 0):
        nqs_set_options(self.h, precision, int(bool(timing)), sample_index_base, energy_tolerance,
                        grad_chunk, audit_samples, tile_blocks_per_sm, table_mb)

    def stage_times(self):
        """{stage: (device ms, kernel launches)} since the previous call."""
        ms = np.zeros(N_STAGES, np.float64)
        nl = np.zeros(N_STAGES, np.int64)
        nqs_stage_times(self.h, ms, nl, N_STAGES)
        return {k: (float(ms[i]), int(nl[i])) for i, k in enumerate(STAGES)}

    def set_system(self, sys_, use_eri=None):
        """Upload the Hamiltonian and ansatz of a workloads.System."""
        h1e = _np(sys_.h1e, np.float64)
        if use_eri is not None:
            nqs_set_hamiltonian(self.h, h1e, _np(use_eri, np.float64), 0, sys_.K, sys_.n_alpha,
                                sys_.n_beta, sys_.e_core)
        else:
            L = _np(sys_.chol, np.float64)
            nqs_set_hamiltonian(self.h, h1e, L, L.shape[0], sys_.K, sys_.n_alpha, sys_.n_beta,
                                sys_.e_core)
        self.K = sys_.K
        self.set_ansatz(sys_.tensors, sys_.pred_ptr, sys_.pred_idx, sys_.rbm_W, sys_.rbm_b)
        rnn = getattr(sys_, "rnn", None)
        if rnn is not None:
            self.set_readout(*rnn)
        if getattr(sys_, "corr", 0):
            self.set_correlator(sys_.corr, getattr(sys_, "rbm_W2", None))
        tk = getattr(sys_, "tucker", None)
        if tk is not None:
            self._keep_tk = (_np(tk[0], np.int32), _np(tk[1], np.float64))
            nqs_set_tensor_term(self.h, self._keep_tk[0], self._keep_tk[1], len(self._keep_tk[1]))

    def set_readout(self, v, eta, w, c, constrained=True):
        """The normalised MPS-RNN / BDG-RNN readout (nqs_set_readout)."""
        self._keep_rnn = tuple(_np(x, np.float64) for x in (v, eta, w, c))
        nqs_set_readout(self.h, *self._keep_rnn, int(bool(constrained)))

    def set_correlator(self, kind, W2=None):
        self._keep_W2 = _np(W2, np.float64)
        nqs_set_correlator(self.h, kind, self._keep_W2)
        self._corr = kind

    def sample(self, n_samples, seed):
        """Autoregressive sampling (nqs_sample): (unique determinants [n][2], counts)."""
        cap = int(min(n_samples, 1 << 20))
        while True:
            s = np.empty((max(cap, 1), 2), np.uint64)
            c = np.empty(max(cap, 1), np.float64)
            try:
                n = nqs_sample(self.h, n_samples, seed, s, c, cap)
                return s[:n], c[:n]
            except NQSError as e:
                if getattr(e, "n_unique", 0) > cap:
                    cap = e.n_unique
                    continue
                raise

    def energy_gradient(self, samples, counts, eps, n_draws, seed, reweighted=False):
        """(grad_sites, grad_W, grad_b, grad_W2, e_loc, summary) of nqs_energy_gradient."""
        s = _np(samples, np.uint64).reshape(-1, 2)
        c = _np(counts, np.float64)
        gT = np.empty((self.n_edges, 4, self.D, self.D), np.float64) if getattr(self, "_keep_rnn", None) is None \
            else None
        gW = np.empty((self.n_hidden, 2 * self.K), np.float64) if self.n_hidden else None
        gb = np.empty(self.n_hidden, np.float64) if self.n_hidden else None
        gW2 = np.empty((self.n_hidden, 2 * self.K, 2 * self.K), np.float64) \
            if self.n_hidden and getattr(self, "_corr", 0) == NQS_CORR_ISING else None
        e = np.empty(len(s), np.float64)
        summ = EnergySummary()
        nqs_energy_gradient(self.h, s, c, len(s), eps, n_draws, seed, reweighted, gT, gW, gb, gW2, e, summ)
        return gT, gW, gb, gW2, e, summ.as_dict()

    def set_ansatz(self, tensors, pred_ptr=None, pred_idx=None, W=None, b=None):
        T = tensors if hasattr(tensors, "data_ptr") else _np(tensors, np.float64)
        self.n_edges, self.D = int(T.shape[0]), int(T.shape[-1])
        self.n_hidden = 0 if W is None else int(W.shape[0])
        self._keep = (T, _np(pred_ptr, np.int32), _np(pred_idx, np.int32),
                      W if (W is None or hasattr(W, "data_ptr")) else _np(W, np.float64),
                      b if (b is None or hasattr(b, "data_ptr")) else _np(b, np.float64))
        T, pp, pi, Wc, bc = self._keep
        nqs_set_ansatz(self.h, T, self.n_edges, self.D, pp, pi, Wc, bc, self.n_hidden)
        self._keep_rnn = None           # the library resets the readout and correlator kind
        self._corr = NQS_CORR_COSH

    def connected(self, samples, eps=0.0):
        """Host-side lists: (offsets, rank, dets, H, sign) as numpy arrays."""
        s = _np(samples, np.uint64).reshape(-1, 2)
        Ns = len(s)
        off = np.zeros(Ns + 1, np.int64)
        nqs_connected(self.h, s, Ns, eps, off, None, None, None, None, 0)
        n = int(off[-1])
        rank = np.empty(max(n, 1), np.uint32)
        dets = np.empty((max(n, 1), 2), np.uint64)
        H = np.empty(max(n, 1), np.float64)
        sg = np.empty(max(n, 1), np.int8)
        nqs_connected(self.h, s, Ns, eps, off, rank, dets, H, sg, n)
        return off, rank[:n], dets[:n], H[:n], sg[:n]

    def amplitude(self, dets):
        d = _np(dets, np.uint64).reshape(-1, 2)
        la = np.empty(len(d), np.float64)
        sg = np.empty(len(d), np.int8)
        nqs_amplitude(self.h, d, len(d), la, sg)
        return la, sg

    def draws(self, samples, eps, n_draws, seed):
        s = _np(samples, np.uint64).reshape(-1, 2)
        r = np.empty((len(s), max(n_draws, 1)), np.int64)
        w = np.empty(len(s), np.uint64)
        nqs_draws(self.h, s, len(s), eps, n_draws, seed, r, w)
        return r[:, :n_draws], w

    def local_energy(self, samples, counts=None, eps=0.0, n_draws=0, seed=0, out=None):
        """E_loc per sample and the summary. `samples` / `counts` / `out` may be
        CUDA tensors (no host copies) or host arrays."""
        if hasattr(samples, "data_ptr"):
            Ns = int(samples.shape[0])
            s = samples
        else:
            s = _np(samples, np.uint64).reshape(-1, 2)
            Ns = len(s)
        c = counts if (counts is None or hasattr(counts, "data_ptr")) else _np(counts, np.float64)
        e = out if out is not None else np.empty(Ns, np.float64)
        summ = EnergySummary()
        nqs_local_energy(self.h, s, c, Ns, eps, n_draws, seed, e, summ)
        return e, summ.as_dict()

    def grad_log_psi_vjp(self, samples, u):
        s = _np(samples, np.uint64).reshape(-1, 2)
        uu = _np(u, np.float64)
        gT = np.empty((self.n_edges, 4, self.D, self.D), np.float64)
        gW = np.empty((self.n_hidden, 2 * self.K), np.float64) if self.n_hidden else None
        gb = np.empty(self.n_hidden, np.float64) if self.n_hidden else None
        nqs_grad_log_psi_vjp(self.h, s, uu, len(s), gT, gW, gb)
        return gT, gW, gb


def local_energy_batch(contexts, args, n_workers=0):
    """E_loc of independent systems in one nqs_local_energy_batch call.

    contexts: one Context per system (each on its own stream for overlap);
    args: per system a dict with samples, counts (or None), eps, n_draws, seed
    (host arrays or CUDA tensors) and optionally out (E_loc destination, host
    array or CUDA tensor). Returns [(e_loc, summary dict)]."""
    n = len(contexts)
    items = (BatchItem * n)()
    keep, outs, sums, grads = [], [], [], []
    for i, (ctx, a) in enumerate(zip(contexts, args)):
        smp = a["samples"]
        if not hasattr(smp, "data_ptr"):
            smp = _np(smp, np.uint64).reshape(-1, 2)
        cnt = a.get("counts")
        if cnt is not None and not hasattr(cnt, "data_ptr"):
            cnt = _np(cnt, np.float64)
        ns = int(smp.shape[0])
        e = a.get("out")
        if e is None:
            e = np.empty(ns, np.float64)
        sm = EnergySummary()
        keep += [smp, cnt]
        outs.append(e)
        sums.append(sm)
        it = items[i]
        it.samples = _ptr(smp)
        it.counts = _ptr(cnt)
        it.n_samples = ns
        it.det_threshold = float(a.get("eps", 0.0))
        it.n_draws = int(a.get("n_draws", 0))
        it.philox_seed = int(a.get("seed", 0))
        it.e_loc = _ptr(e)
        it.summary = C.pointer(sm)
        if a.get("grad"):
            # energy gradient of this system: site tensors, and W, b with a correlator
            gT = np.empty((ctx.n_edges, 4, ctx.D, ctx.D), np.float64)
            gW = np.empty((ctx.n_hidden, 2 * ctx.K), np.float64) if ctx.n_hidden else None
            gb = np.empty(ctx.n_hidden, np.float64) if ctx.n_hidden else None
            grads.append((gT, gW, gb))
            it.reweighted = int(bool(a.get("reweighted", False)))
            it.grad_sites, it.grad_W, it.grad_b = _ptr(gT), _ptr(gW), _ptr(gb)
        else:
            grads.append(None)
    nqs_local_energy_batch([c.h for c in contexts], items, n_workers)
    return [(e, sm.as_dict()) if g is None else (e, sm.as_dict(), g)
            for e, sm, g in zip(outs, sums, grads)]


_LOG_PSI = None


def log_psi(context, samples, tensors, W=None, b=None, pred_ptr=None, pred_idx=None):
    """log|psi(n)| (and the sign) as a differentiable function of the ansatz
    parameters: forward is nqs_amplitude, backward nqs_grad_log_psi_vjp (the
    hand-written reverse sweep of Eq. egrad's d ln psi / d theta).

    tensors [n_edges][4][D][D], W [n_hidden][2K], b [n_hidden]: torch tensors
    (CUDA or CPU; gradients come back on the same device and dtype). The
    context must hold the system's Hamiltonian and run on the current torch
    stream (the default of Context). Returns (log_abs [Ns] float64, sign [Ns]
    int8, not differentiable)."""
    global _LOG_PSI
    if _LOG_PSI is None:
        _LOG_PSI = _make_log_psi()
    return _LOG_PSI.apply(context, samples, tensors, W, b, pred_ptr, pred_idx)


def _make_log_psi():
    import torch

    def upload(context, T, W, b, pp, pi):
        context.set_ansatz(T, pp, pi, W, b)
        context._ansatz_token = object()
        return context._ansatz_token

    def f64(x):
        return None if x is None else x.detach().to(torch.float64).contiguous()

    class LogPsi(torch.autograd.Function):
        @staticmethod
        def forward(fctx, context, samples, tensors, W, b, pred_ptr, pred_idx):
            T, Wd, bd = f64(tensors), f64(W), f64(b)
            token = upload(context, T, Wd, bd, pred_ptr, pred_idx)
            s = samples if hasattr(samples, "data_ptr") else torch.from_numpy(
                _np(samples, np.uint64).reshape(-1, 2).view(np.int64))
            s = s.to(T.device).contiguous()
            Ns = int(s.shape[0])
            la = torch.empty(Ns, dtype=torch.float64, device=T.device)
            sg = torch.empty(Ns, dtype=torch.int8, device=T.device)
            nqs_amplitude(context.h, s, Ns, la, sg)
            fctx.context, fctx.token, fctx.graph = context, token, (pred_ptr, pred_idx)
            fctx.dtypes = (tensors.dtype, None if W is None else W.dtype, None if b is None else b.dtype)
            fctx.save_for_backward(s, T, *( [Wd, bd] if Wd is not None else []))
            fctx.mark_non_differentiable(sg)
            return la, sg

        @staticmethod
        def backward(fctx, g_la, g_sg):
            saved = fctx.saved_tensors
            s, T = saved[0], saved[1]
            Wd, bd = (saved[2], saved[3]) if len(saved) > 2 else (None, None)
            context = fctx.context
            if getattr(context, "_ansatz_token", None) is not fctx.token:
                upload(context, T, Wd, bd, *fctx.graph)   # parameters changed since forward
            u = g_la.detach().to(device=T.device, dtype=torch.float64).contiguous()
            gT = torch.empty_like(T)
            gW = torch.empty_like(Wd) if Wd is not None else None
            gb = torch.empty_like(bd) if bd is not None else None
            nqs_grad_log_psi_vjp(context.h, s, u, int(s.shape[0]), gT, gW, gb)
            dt, dw, db = fctx.dtypes
            return (None, None, gT.to(dt), None if gW is None else gW.to(dw),
                    None if gb is None else gb.to(db), None, None)

    return LogPsi
