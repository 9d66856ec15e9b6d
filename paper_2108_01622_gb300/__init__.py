"""GB300 loop-hafnian library (arXiv:2108.01622): thin Python binding of include/lhaf.h.

Argument marshalling only: every step of the computation runs in the CUDA library
``liblhaf_gb300.so`` built in-tree by ``paper_2108_01622_gb300.build``. There is no CPU fallback;
if the library is missing, every call raises ImportError.

Inputs may be numpy arrays (host pointers: synchronous calls) or torch CUDA tensors (device
pointers: calls ordered on the context's stream, which defaults to torch's current stream).
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblhaf_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "lhaf.h")

DEVICE_PTRS = 0x1
FP32_TERMS = 0x2
PLAIN_ACCUM = 0x4
NO_REPEAT_SPEEDUP = 0x8
NO_LOOPS = 0x10
BATCH_B_PER_ITEM = 0x20
NO_ZERO_SPLIT = 0x40
ET = 0x80  # eigenvalue-trace inclusion/exclusion instead of the finite difference sieve

STATUS = {0: "LHAF_OK", 1: "LHAF_EINVAL", 2: "LHAF_ETOOBIG", 3: "LHAF_ECUDA", 4: "LHAF_ETIMEOUT",
          5: "LHAF_ENOMEM", 6: "LHAF_ECANCELLED"}


class LhafError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        detail = _lib().lhaf_last_error().decode() if status == 3 else ""
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_lib().lhaf_strerror(status).decode()})"
                         + (f" [{detail}]" if detail else ""))


class Stats(ctypes.Structure):
    _fields_ = [("terms", ctypes.c_uint64), ("n_dim", ctypes.c_int32), ("h", ctypes.c_int32),
                ("pairs", ctypes.c_int32), ("team", ctypes.c_int32), ("kernel_ms", ctypes.c_double),
                ("flops_model", ctypes.c_double), ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
                ("launches", ctypes.c_int32), ("term_launches", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2108_01622_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        vp, c = ctypes.c_void_p, ctypes
        L.lhaf_ctx_create.argtypes = [ctypes.POINTER(vp), c.c_int, vp]
        L.lhaf_ctx_create.restype = c.c_int
        L.lhaf_ctx_destroy.argtypes = [vp]
        L.lhaf_ctx_destroy.restype = None
        L.lhaf_strerror.argtypes = [c.c_int]
        L.lhaf_strerror.restype = c.c_char_p
        L.lhaf_last_error.argtypes = []
        L.lhaf_last_error.restype = c.c_char_p
        L.lhaf_plan.argtypes = [c.c_int, vp, c.c_uint32, c.c_int, ctypes.POINTER(c.c_uint64),
                                ctypes.POINTER(c.c_int32), ctypes.POINTER(c.c_int32), ctypes.POINTER(c.c_int32)]
        L.lhaf_plan.restype = c.c_int
        L.lhaf_plan_groups.argtypes = [c.c_int, vp, c.c_uint32, c.c_int, ctypes.POINTER(c.c_int32)]
        L.lhaf_plan_groups.restype = c.c_int
        L.lhaf.argtypes = [vp, c.c_int, vp, vp, vp, c.c_uint32, vp, ctypes.POINTER(Stats)]
        L.lhaf.restype = c.c_int
        L.lhaf_range.argtypes = [vp, c.c_int, vp, vp, vp, c.c_uint32, c.c_uint64, c.c_uint64, vp,
                                 ctypes.POINTER(Stats)]
        L.lhaf_range.restype = c.c_int
        L.lhaf_combine.argtypes = [c.c_int, vp, c.c_int32, vp]
        L.lhaf_combine.restype = c.c_int
        L.lhaf_flops_per_term.argtypes = [c.c_int, c.c_int, c.c_int]
        L.lhaf_flops_per_term.restype = c.c_double
        L.lhaf_batched.argtypes = [vp, c.c_int, c.c_int, vp, vp, vp, c.c_uint32, vp, vp, ctypes.POINTER(Stats)]
        L.lhaf_batched.restype = c.c_int
        L.gbs_pattern_prob.argtypes = [vp, c.c_int, vp, vp, vp, vp, c.c_uint32, ctypes.POINTER(c.c_double), vp]
        L.gbs_pattern_prob.restype = c.c_int
        L.gbs_pattern_prob_mixed.argtypes = [vp, c.c_int, vp, vp, vp, c.c_uint32, ctypes.POINTER(c.c_double), vp]
        L.gbs_pattern_prob_mixed.restype = c.c_int
        L.gbs_chain_rule_step.argtypes = [vp, c.c_int, vp, vp, vp, vp, vp, c.c_int, c.c_int, c.c_double,
                                          c.c_uint32, vp, ctypes.POINTER(c.c_int32)]
        L.gbs_chain_rule_step.restype = c.c_int
        L.lhaf_multi_gamma.argtypes = [vp, c.c_int, vp, c.c_int, vp, vp, c.c_uint32, vp, vp]
        L.lhaf_multi_gamma.restype = c.c_int
        L.lhaf_grad.argtypes = [vp, c.c_int, vp, vp, vp, c.c_uint32, vp, vp, vp]
        L.lhaf_grad.restype = c.c_int
        L.lhaf_grad_batched.argtypes = [vp, c.c_int, c.c_int, vp, vp, vp, c.c_uint32, vp, vp, vp, vp]
        L.lhaf_grad_batched.restype = c.c_int
        L.lhaf_batched_plan_create.argtypes = [vp, c.c_int, c.c_int, vp, vp, vp, c.c_uint32, ctypes.POINTER(vp)]
        L.lhaf_batched_plan_create.restype = c.c_int
        L.lhaf_batched_plan_exec.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(Stats)]
        L.lhaf_batched_plan_exec.restype = c.c_int
        L.lhaf_batched_plan_destroy.argtypes = [vp]
        L.lhaf_batched_plan_destroy.restype = None
        L.lhaf_batched_mode.argtypes = [vp, c.c_int, vp, vp, vp, c.c_int, c.c_int, c.c_uint32, vp,
                                        ctypes.POINTER(Stats)]
        L.lhaf_batched_mode.restype = c.c_int
        L.lhaf_fp64_probe.argtypes = [c.c_int, ctypes.POINTER(c.c_double)]
        L.lhaf_fp64_probe.restype = c.c_int
        _LIB = L
    return _LIB


def header_functions() -> list:
    """Names of the functions include/lhaf.h declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                                 src, flags=re.M)))


def _check(st: int, where: str):
    if st != 0:
        raise LhafError(st, where)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _host_c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _reps_arr(reps, M) -> Optional[np.ndarray]:
    if reps is None:
        return None
    r = np.ascontiguousarray(np.asarray(reps, dtype=np.int32))
    if r.shape != (M,):
        raise ValueError(f"reps must have shape ({M},)")
    return r


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    return a.ctypes.data


def plan(reps: Sequence[int], flags: int = 0, has_loops: bool = True) -> Tuple[int, int, int, int]:
    """(terms, n_dim, h, pairs) of the greedy repeated-pair sieve (App. B.3), host only."""
    r = np.ascontiguousarray(np.asarray(reps, dtype=np.int32))
    T, nd, h, P = ctypes.c_uint64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib().lhaf_plan(len(r), r.ctypes.data, flags, int(has_loops), ctypes.byref(T), ctypes.byref(nd),
                            ctypes.byref(h), ctypes.byref(P)), "lhaf_plan")
    return T.value, nd.value, h.value, P.value


def plan_groups(reps: Sequence[int], flags: int = 0, has_loops: bool = True) -> int:
    """Number of zero-digit groups the sieve runs as (0: a single sieve on the full matrix); with ET,
    the number of support sizes."""
    r = np.ascontiguousarray(np.asarray(reps, dtype=np.int32))
    g = ctypes.c_int32()
    _check(_lib().lhaf_plan_groups(len(r), r.ctypes.data, flags, int(has_loops), ctypes.byref(g)), "lhaf_plan_groups")
    return g.value


def flops_per_term(n_dim: int, h: int, bordered: bool) -> float:
    return _lib().lhaf_flops_per_term(n_dim, h, int(bordered))


def fp64_probe(device: int = 0) -> float:
    """Measured FP64 FMA throughput of the device in GFLOP/s."""
    g = ctypes.c_double()
    _check(_lib().lhaf_fp64_probe(device, ctypes.byref(g)), "lhaf_fp64_probe")
    return g.value


def combine(partials, h: int) -> complex:
    p = np.ascontiguousarray(np.asarray(partials, dtype=np.float64).reshape(-1, 4))
    out = np.zeros(1, np.complex128)
    _check(_lib().lhaf_combine(p.shape[0], p.ctypes.data, h, out.ctypes.data), "lhaf_combine")
    return complex(out[0])


class Context:
    """A device context: stream, workspace and the lhaf entry points."""

    def __init__(self, device: int = 0, stream=None):
        self._lib = _lib()
        self.device = device
        if stream is None:
            try:
                import torch

                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except ImportError:
                pass
        if stream == 0:
            # torch's default stream is the legacy default stream (handle 0), which the library would
            # read as "create a private stream": pass cudaStreamLegacy instead so that work is ordered
            # with torch's own kernels and events
            stream = 1
        self.stream = stream
        h = ctypes.c_void_p()
        _check(self._lib.lhaf_ctx_create(ctypes.byref(h), device, stream), "lhaf_ctx_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lhaf_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _inputs(self, B, gamma, reps, flags):
        dev = _is_torch(B) and B.is_cuda
        if dev:
            import torch

            if B.dtype != torch.complex128:
                raise TypeError("B must be complex128")
            B = B.contiguous()
            if gamma is not None:
                gamma = gamma.to(torch.complex128).contiguous()
            flags |= DEVICE_PTRS
        else:
            B = _host_c128(B)
            gamma = None if gamma is None else _host_c128(gamma)
        M = B.shape[0]
        if tuple(B.shape) != (M, M):
            raise ValueError("B must be square")
        if gamma is not None and tuple(gamma.shape) != (M,):
            raise ValueError("gamma must have shape (M,)")
        return B, gamma, _reps_arr(reps, M), M, flags

    def lhaf(self, B, gamma=None, reps=None, flags: int = 0, stats: bool = False, out=None):
        """lhaf(B_n). Host inputs return a Python complex. Device (torch CUDA) inputs write into
        `out` (a complex128 CUDA tensor of one element, allocated if None) and return it."""
        B, gamma, r, M, flags = self._inputs(B, gamma, reps, flags)
        st = Stats()
        if flags & DEVICE_PTRS:
            import torch

            if out is None:
                out = torch.empty(1, dtype=torch.complex128, device=B.device)
            _check(self._lib.lhaf(self._h, M, _ptr(B), _ptr(gamma), _ptr(r), flags, out.data_ptr(),
                                  ctypes.byref(st) if stats else None), "lhaf")
            return (out, st.as_dict()) if stats else out
        res = np.zeros(1, np.complex128)
        _check(self._lib.lhaf(self._h, M, _ptr(B), _ptr(gamma), _ptr(r), flags, res.ctypes.data,
                              ctypes.byref(st) if stats else None), "lhaf")
        return (complex(res[0]), st.as_dict()) if stats else complex(res[0])

    def lhaf_range(self, B, gamma, reps, term_begin: int, term_end: int, flags: int = 0, stats: bool = False):
        """Unscaled double-double partial (4 doubles) of the sieve over [term_begin, term_end)."""
        B, gamma, r, M, flags = self._inputs(B, gamma, reps, flags)
        st = Stats()
        if flags & DEVICE_PTRS:
            import torch

            part = torch.zeros(4, dtype=torch.float64, device=B.device)
            _check(self._lib.lhaf_range(self._h, M, _ptr(B), _ptr(gamma), _ptr(r), flags, term_begin, term_end,
                                        part.data_ptr(), ctypes.byref(st) if stats else None), "lhaf_range")
        else:
            part = np.zeros(4, np.float64)
            _check(self._lib.lhaf_range(self._h, M, _ptr(B), _ptr(gamma), _ptr(r), flags, term_begin, term_end,
                                        part.ctypes.data, ctypes.byref(st) if stats else None), "lhaf_range")
        return (part, st.as_dict()) if stats else part

    def lhaf_batched(self, B, gammas, reps, flags: int = 0, stats: bool = False, out=None):
        """Loop hafnians of a batch: item i uses reps[i] and gammas[i] (batch x M; None for diag(B))
        with the shared M x M matrix B (or batch x M x M with BATCH_B_PER_ITEM). Host inputs return
        (values, item_status) as numpy arrays; torch CUDA inputs write `out` (complex128, batch)."""
        dev = _is_torch(B) and B.is_cuda
        r = np.ascontiguousarray(np.asarray(reps, dtype=np.int32))
        if r.ndim != 2:
            raise ValueError("reps must be batch x M")
        batch, M = r.shape
        st = Stats()
        status = np.zeros(batch, dtype=np.int32)
        if dev:
            import torch

            flags |= DEVICE_PTRS
            B = B.to(torch.complex128).contiguous()
            g = None if gammas is None else gammas.to(torch.complex128).contiguous()
            if out is None:
                out = torch.empty(batch, dtype=torch.complex128, device=B.device)
            _check(self._lib.lhaf_batched(self._h, batch, M, B.data_ptr(), None if g is None else g.data_ptr(),
                                          r.ctypes.data, flags, out.data_ptr(), status.ctypes.data,
                                          ctypes.byref(st) if stats else None), "lhaf_batched")
            res = out
        else:
            Bh = _host_c128(B)
            gh = None if gammas is None else _host_c128(gammas)
            res = np.zeros(batch, np.complex128)
            _check(self._lib.lhaf_batched(self._h, batch, M, Bh.ctypes.data, None if gh is None else gh.ctypes.data,
                                          r.ctypes.data, flags, res.ctypes.data, status.ctypes.data,
                                          ctypes.byref(st) if stats else None), "lhaf_batched")
        if stats:
            return res, status, st.as_dict()
        return res, status

    def batched_plan(self, B, gammas, reps, flags: int = 0) -> "BatchedPlan":
        """A BatchedPlan for the patterns `reps` (batch x M): planned, tuned on (B, gammas) and
        captured in a CUDA graph once; BatchedPlan.run evaluates new values of B and gammas."""
        return BatchedPlan(self, B, gammas, reps, flags)

    def lhaf_batched_mode(self, B, gamma, reps, mode: int, n_cut: int, flags: int = 0, stats: bool = False):
        """lhaf(B_{reps + n e_mode}) for n = 0..n_cut (reps[mode] == 0) with shared sieve terms
        (App. B.5). Host inputs; returns a complex128 array of n_cut + 1 values."""
        Bh = _host_c128(B)
        M = Bh.shape[0]
        gh = None if gamma is None else _host_c128(gamma)
        r = _reps_arr(reps, M)
        out = np.zeros(n_cut + 1, np.complex128)
        st = Stats()
        _check(self._lib.lhaf_batched_mode(self._h, M, Bh.ctypes.data, None if gh is None else gh.ctypes.data,
                                           r.ctypes.data, mode, n_cut, flags, out.ctypes.data,
                                           ctypes.byref(st) if stats else None), "lhaf_batched_mode")
        return (out, st.as_dict()) if stats else out

    def gbs_pattern_prob(self, U, r, alpha, n, flags: int = 0):
        """(P(n), lhaf(B_n)) for the pure state (U, r, alpha) (App. A, Eq. mixed_prob)."""
        Uh = _host_c128(U)
        M = Uh.shape[0]
        rh = np.ascontiguousarray(np.asarray(r, dtype=np.float64))
        ah = None if alpha is None else _host_c128(alpha)
        nh = _reps_arr(n, M)
        prob = ctypes.c_double()
        lh = np.zeros(1, np.complex128)
        _check(self._lib.gbs_pattern_prob(self._h, M, Uh.ctypes.data, rh.ctypes.data,
                                          None if ah is None else ah.ctypes.data, nh.ctypes.data, flags,
                                          ctypes.byref(prob), lh.ctypes.data), "gbs_pattern_prob")
        return prob.value, complex(lh[0])

    def gbs_pattern_prob_mixed(self, sigma, alpha, n, flags: int = 0):
        """(P(n), lhaf(A_n)) for the Gaussian state with complex covariance sigma (2M x 2M) and mean
        alpha (App. A, Eq. mixed_prob), mixed (lossy) states included."""
        S = _host_c128(sigma)
        M = S.shape[0] // 2
        ah = None if alpha is None else _host_c128(alpha)
        nh = _reps_arr(n, M)
        prob = ctypes.c_double()
        lh = np.zeros(1, np.complex128)
        _check(self._lib.gbs_pattern_prob_mixed(self._h, M, S.ctypes.data, None if ah is None else ah.ctypes.data,
                                                nh.ctypes.data, flags, ctypes.byref(prob), lh.ctypes.data),
               "gbs_pattern_prob_mixed")
        return prob.value, complex(lh[0])

    def gbs_chain_rule_step(self, U, r, alpha, beta, n, mode: int, n_cut: int, u: float = -1.0, flags: int = 0):
        """(cond, drawn): the distribution of the photon number of `mode` (0..n_cut) given the photon
        numbers n and the coherent amplitudes beta of the other modes (App. A.2), and the outcome drawn
        with the uniform number u (-1 when u is outside [0, 1))."""
        Uh = _host_c128(U)
        M = Uh.shape[0]
        rh = np.ascontiguousarray(np.asarray(r, dtype=np.float64))
        ah = None if alpha is None else _host_c128(alpha)
        bh = None if beta is None else _host_c128(beta)
        nh = _reps_arr(n, M)
        cond = np.zeros(n_cut + 1, np.float64)
        drawn = ctypes.c_int32(-1)
        _check(self._lib.gbs_chain_rule_step(self._h, M, Uh.ctypes.data, rh.ctypes.data,
                                             None if ah is None else ah.ctypes.data,
                                             None if bh is None else bh.ctypes.data, nh.ctypes.data, int(mode),
                                             int(n_cut), float(u), flags, cond.ctypes.data, ctypes.byref(drawn)),
               "gbs_chain_rule_step")
        return cond, drawn.value

    def lhaf_multi_gamma(self, B, gammas, reps, flags: int = 0, stats: bool = False):
        """lhaf(B_n) for each row of gammas (loop weights), sharing every sieve term's reduction and
        characteristic polynomial (App. B.5, threshold sub-detectors)."""
        Bh = _host_c128(B)
        M = Bh.shape[0]
        G = _host_c128(gammas).reshape(-1, M)
        G = np.ascontiguousarray(G)
        rh = _reps_arr(reps, M)
        out = np.zeros(G.shape[0], np.complex128)
        st = Stats()
        _check(self._lib.lhaf_multi_gamma(self._h, M, Bh.ctypes.data, G.shape[0], G.ctypes.data, rh.ctypes.data,
                                          flags, out.ctypes.data, ctypes.byref(st) if stats else None),
               "lhaf_multi_gamma")
        return (out, st.as_dict()) if stats else out

    def lhaf_grad(self, B, gamma=None, reps=None, flags: int = 0):
        """(lhaf(B_n), dB (M x M, symmetric-variable derivative), dgamma (M,) or None)."""
        Bh = _host_c128(B)
        M = Bh.shape[0]
        gh = None if gamma is None else _host_c128(gamma)
        r = _reps_arr(reps, M)
        val = np.zeros(1, np.complex128)
        dB = np.zeros((M, M), np.complex128)
        dg = np.zeros(M, np.complex128)
        _check(self._lib.lhaf_grad(self._h, M, Bh.ctypes.data, None if gh is None else gh.ctypes.data, _ptr(r), flags,
                                   val.ctypes.data, dB.ctypes.data, dg.ctypes.data), "lhaf_grad")
        return complex(val[0]), dB, (None if gh is None else dg)

    def lhaf_grad_batched(self, B, gammas, reps, flags: int = 0):
        """Values (batch,), dB (batch x M x M), dgamma (batch x M, or None when gammas is None) and
        item statuses of the loop hafnians of `reps` (batch x M) with the shared matrix B."""
        Bh = _host_c128(B)
        M = Bh.shape[0]
        r = np.ascontiguousarray(np.asarray(reps, dtype=np.int32))
        if r.ndim != 2 or r.shape[1] != M:
            raise ValueError("reps must be batch x M")
        batch = r.shape[0]
        gh = None if gammas is None else np.ascontiguousarray(np.asarray(gammas, dtype=np.complex128).reshape(batch, M))
        vals = np.zeros(batch, np.complex128)
        dB = np.zeros((batch, M, M), np.complex128)
        dg = np.zeros((batch, M), np.complex128)
        st = np.zeros(batch, np.int32)
        _check(self._lib.lhaf_grad_batched(self._h, batch, M, Bh.ctypes.data, None if gh is None else gh.ctypes.data,
                                           r.ctypes.data, flags, vals.ctypes.data, dB.ctypes.data, dg.ctypes.data,
                                           st.ctypes.data), "lhaf_grad_batched")
        return vals, dB, (None if gh is None else dg), st


class BatchedPlan:
    """lhaf_batched for fixed patterns, replayed from a captured CUDA graph (include/lhaf.h,
    lhaf_batched_plan_*). Inputs are numpy arrays (host) or torch CUDA tensors (device), as chosen
    at creation; B and gammas keep their creation shapes."""

    def __init__(self, ctx: Context, B, gammas, reps, flags: int = 0):
        self._ctx = ctx
        self._lib = ctx._lib
        r = np.ascontiguousarray(np.asarray(reps, dtype=np.int32))
        if r.ndim != 2:
            raise ValueError("reps must be batch x M")
        self.batch, self.M = r.shape
        self.dev = _is_torch(B) and B.is_cuda
        self.with_gamma = gammas is not None
        if self.dev:
            flags |= DEVICE_PTRS
        self.flags = flags
        Bp, gp, keep = self._marshal(B, gammas)
        h = ctypes.c_void_p()
        _check(self._lib.lhaf_batched_plan_create(ctx._h, self.batch, self.M, Bp, gp, r.ctypes.data, flags,
                                                  ctypes.byref(h)), "lhaf_batched_plan_create")
        del keep
        self._h = h

    def _marshal(self, B, gammas):
        if (gammas is not None) != self.with_gamma:
            raise ValueError("gammas must be given exactly when they were given at creation")
        if self.dev:
            import torch

            Bt = B.to(torch.complex128).contiguous()
            gt = None if gammas is None else gammas.to(torch.complex128).contiguous()
            return Bt.data_ptr(), (None if gt is None else gt.data_ptr()), (Bt, gt)
        Bh = _host_c128(B)
        gh = None if gammas is None else _host_c128(gammas)
        return Bh.ctypes.data, (None if gh is None else gh.ctypes.data), (Bh, gh)

    def run(self, B, gammas=None, stats: bool = False, out=None):
        """Values of the batch for new B and gammas: (values, item_status[, stats])."""
        if not getattr(self, "_h", None):
            raise RuntimeError("plan is closed")
        Bp, gp, keep = self._marshal(B, gammas)
        st = Stats()
        status = np.zeros(self.batch, dtype=np.int32)
        if self.dev:
            import torch

            if out is None:
                out = torch.empty(self.batch, dtype=torch.complex128, device=B.device)
            res, optr = out, out.data_ptr()
        else:
            res = np.zeros(self.batch, np.complex128)
            optr = res.ctypes.data
        _check(self._lib.lhaf_batched_plan_exec(self._h, Bp, gp, optr, status.ctypes.data,
                                                ctypes.byref(st) if stats else None), "lhaf_batched_plan_exec")
        del keep
        return (res, status, st.as_dict()) if stats else (res, status)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lhaf_batched_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
