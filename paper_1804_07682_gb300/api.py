"""Python binding of libgnaosc.so: argument marshalling over the C ABI.

PyTorch supplies device memory and the current CUDA stream; every step of the
chain runs in the library's kernels.  There is no CPU path: if the library is
missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _native as N

PRECISIONS = {"fp64": N.GNA_FP64, "f64phase": N.GNA_MIXED_F64PHASE, "ff": N.GNA_MIXED_FFPHASE}
KINDS = {"pearson": N.GNA_PEARSON, "poisson": N.GNA_POISSON, 0: N.GNA_PEARSON, 1: N.GNA_POISSON}


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr_any(t: torch.Tensor):
    """Pointer to a CUDA tensor or to pinned host memory (mapped into the device's
    address space: kernels read and write it in place)."""
    if not (t.is_cuda or t.is_pinned()):
        raise ValueError("expected a CUDA tensor or pinned host memory")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("the oscillation library needs a CUDA device")
    N.lib()


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def gl_nodes(n: int, device="cuda"):
    """n-point Gauss-Legendre nodes (ascending) and weights on [-1, 1], computed on the device."""
    _require_cuda()
    x = torch.empty(n, dtype=torch.float64, device=device)
    w = torch.empty(n, dtype=torch.float64, device=device)
    N.check(N.lib().gna_gl_nodes(int(n), _ptr(x), _ptr(w), ctypes.c_void_p(_stream())), what="gna_gl_nodes")
    return x, w


def _oscprob_out(E: torch.Tensor, nL: int, prec: str, out: Optional[torch.Tensor]) -> torch.Tensor:
    """Output of the element-wise calls: on E's device, or, for E in pinned host
    memory (read by the kernel in place over the host link), in pinned host memory."""
    out_dtype = torch.float64 if prec == "fp64" else torch.float32
    if out is not None:
        if out.dtype != out_dtype or tuple(out.shape) != (nL, E.numel()):
            raise ValueError("out must be %s [%d, %d]" % (out_dtype, nL, E.numel()))
        if not out.is_cuda and not out.is_pinned():
            raise ValueError("a host output must be pinned")
        return out
    if E.is_cuda:
        return torch.empty((nL, E.numel()), dtype=out_dtype, device=E.device)
    if not E.is_pinned():
        raise ValueError("E must be a CUDA tensor or pinned host memory")
    return torch.empty((nL, E.numel()), dtype=out_dtype).pin_memory()


def oscprob(E: torch.Tensor, L: Sequence[float], theta: Sequence[float], prec: str = "fp64",
            out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Element-wise OscProb: P(nue_bar -> nue_bar) [nL, n] at energies E (MeV) for baselines L (km).
    E and out may be CUDA tensors or pinned host memory (the kernel reads and writes it in place)."""
    _require_cuda()
    if E.dtype != torch.float64:
        raise ValueError("E must be float64")
    if not E.is_cuda and not E.is_pinned():
        raise ValueError("E must be a CUDA tensor or pinned host memory")
    Ls = _f64(L)
    p = N.GnaOsc(*[float(t) for t in theta])
    P = _oscprob_out(E, Ls.size, prec, out)
    code = N.lib().gna_oscprob_ee(_ptr_any(E), E.numel(), Ls.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  Ls.size, ctypes.byref(p), PRECISIONS[prec], _ptr_any(P), ctypes.c_void_p(_stream()))
    N.check(code, what="gna_oscprob_ee")
    return P


def oscprob_staged(E: torch.Tensor, L: Sequence[float], theta: Sequence[float], prec: str = "fp64",
                   out: Optional[torch.Tensor] = None, chunk: int = 0) -> torch.Tensor:
    """OscProb from pinned host E to pinned host P [nL, n] through device staging
    buffers, chunk by chunk, with the transfers overlapping the evaluation
    (gna_oscprob_ee_staged).  Ordered on the current stream: P is complete once
    that stream has synchronised."""
    _require_cuda()
    if E.dtype != torch.float64:
        raise ValueError("E must be float64")
    if E.is_cuda or not E.is_pinned():
        raise ValueError("E must be pinned host memory")
    Ls = _f64(L)
    p = N.GnaOsc(*[float(t) for t in theta])
    P = _oscprob_out(E, Ls.size, prec, out)
    if P.is_cuda:
        raise ValueError("out must be pinned host memory")
    code = N.lib().gna_oscprob_ee_staged(_ptr_any(E), E.numel(), Ls.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         Ls.size, ctypes.byref(p), PRECISIONS[prec], _ptr_any(P), int(chunk),
                                         ctypes.c_void_p(_stream()))
    N.check(code, what="gna_oscprob_ee_staged")
    return P


FLAVOURS = {"e": 0, "mu": 1, "tau": 2}


def pmns(theta_full: Sequence[float]) -> np.ndarray:
    """Mixing matrix U[alpha][i] (complex 3x3, host) for (s2_12, s2_13, s2_23, delta_cp, dm2_21, dm2_32)."""
    p = N.GnaOscFull(*[float(t) for t in theta_full])
    re = np.empty(9)
    im = np.empty(9)
    P = ctypes.POINTER(ctypes.c_double)
    N.check(N.lib().gna_pmns(ctypes.byref(p), re.ctypes.data_as(P), im.ctypes.data_as(P)), what="gna_pmns")
    return (re + 1j * im).reshape(3, 3)


def oscprob_general(E: torch.Tensor, L: Sequence[float], theta_full: Sequence[float], alpha="mu", beta="e",
                    anti: bool = False, prec: str = "fp64", out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Element-wise OscProb for any channel: P(alpha -> beta) [nL, n] at energies E (MeV) for
    baselines L (km); theta_full = (s2_12, s2_13, s2_23, delta_cp, dm2_21, dm2_32).  E and out
    may be CUDA tensors or pinned host memory."""
    _require_cuda()
    if E.dtype != torch.float64:
        raise ValueError("E must be float64")
    if not E.is_cuda and not E.is_pinned():
        raise ValueError("E must be a CUDA tensor or pinned host memory")
    a = FLAVOURS.get(alpha, alpha)
    b = FLAVOURS.get(beta, beta)
    Ls = _f64(L)
    p = N.GnaOscFull(*[float(t) for t in theta_full])
    P = _oscprob_out(E, Ls.size, prec, out)
    code = N.lib().gna_oscprob(_ptr_any(E), E.numel(), Ls.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               Ls.size, int(a), int(b), int(bool(anti)), ctypes.byref(p), PRECISIONS[prec], _ptr_any(P),
                               ctypes.c_void_p(_stream()))
    N.check(code, what="gna_oscprob")
    return P


def poisson_datasets(mu, ndatasets: int, seed: int, stream=None) -> torch.Tensor:
    """Poisson pseudo-data [ndatasets, nbins] (float64, CUDA) of the bin means mu
    (host, each in [0, 700]), reproducible from the seed (counter-based)."""
    _require_cuda()
    m = _f64(mu)
    out = torch.empty((int(ndatasets), m.size), dtype=torch.float64, device="cuda")
    code = N.lib().gna_poisson_datasets(m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), m.size, int(ndatasets),
                                        ctypes.c_uint64(int(seed)), _ptr(out), ctypes.c_void_p(_stream(stream)))
    N.check(code, what="gna_poisson_datasets")
    return out


def fp32_probe(blocks: int, iters: int, out: Optional[torch.Tensor] = None, stream=None) -> int:
    """Enqueues the FP32 FMA-rate probe (blocks x 256 threads, 8 chains of
    iters FMAs each) on the current stream; returns the FMAs it executes."""
    _require_cuda()
    if out is None:
        out = torch.empty(1, dtype=torch.float32, device="cuda")
    N.check(N.lib().gna_fp32_probe(int(blocks), int(iters), _ptr(out), ctypes.c_void_p(_stream(stream))),
            what="gna_fp32_probe")
    return int(blocks) * 256 * 8 * int(iters)


class Plan:
    """A configured chain (paper's configuration stage): energy grids built and
    all scratch allocated on the device; evaluations only launch kernels."""

    def __init__(self, edges, L, nodes_per_bin: int = 0, npts: int = 1, node_counts=None, Lweight=None,
                 norm: float = 1.0, e_scale: float = 1.0, prec: str = "ff", kind="pearson", max_datasets: int = 0,
                 with_plain: bool = False, mapping: Optional[str] = None, channel=None, stream=None):
        """channel: None for the nue_bar survival chain (``eval``), or (alpha, beta,
        anti) with flavours "e", "mu", "tau" for the chain of P(alpha -> beta)
        (``eval_general``, parameters (s2_12, s2_13, s2_23, delta_cp, dm2_21, dm2_32))."""
        _require_cuda()
        self._lib = N.lib()
        self._edges = _f64(edges)
        self._L = _f64(np.atleast_1d(L))
        self._Lw = None if Lweight is None else _f64(Lweight)
        self._counts = None if node_counts is None else np.ascontiguousarray(np.asarray(node_counts, dtype=np.int32))
        self.nbins = self._edges.size - 1
        self.npts = int(npts)
        self.nL = self._L.size
        self.prec = prec
        flags = N.GNA_PLAN_WITH_PLAIN if with_plain else 0
        if mapping == "split":
            flags |= N.GNA_PLAN_FORCE_SPLIT
        elif mapping == "bins":
            flags |= N.GNA_PLAN_FORCE_BINS
        elif mapping == "slices":
            flags |= N.GNA_PLAN_FORCE_SLICES
        elif mapping is not None:
            raise ValueError("mapping must be 'split', 'bins', 'slices' or None")
        self.channel = None
        if channel is not None:
            a, b, anti = channel
            self.channel = (FLAVOURS[a], FLAVOURS[b], int(bool(anti)))
            flags |= N.GNA_PLAN_GENERAL
        P = ctypes.POINTER(ctypes.c_double)
        d = N.GnaPlanDesc()
        d.nbins = self.nbins
        d.edges = self._edges.ctypes.data_as(P)
        d.nodes_per_bin = int(nodes_per_bin)
        d.npts = self.npts
        d.node_counts = None if self._counts is None else self._counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.nL = self.nL
        d.L = self._L.ctypes.data_as(P)
        d.Lweight = None if self._Lw is None else self._Lw.ctypes.data_as(P)
        d.norm = float(norm)
        d.e_scale = float(e_scale)
        d.prec = PRECISIONS[prec]
        d.kind = KINDS[kind]
        d.max_datasets = int(max_datasets)
        d.flags = flags
        if self.channel is not None:
            d.alpha, d.beta, d.anti = self.channel
        h = ctypes.c_void_p()
        code = self._lib.gna_plan_create(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(_stream(stream)))
        N.check(code, what="gna_plan_create")
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._scratch = {}

    # ------------------------------------------------------------ basics --
    def close(self):
        if getattr(self, "_h", None):
            self._lib.gna_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, code, what):
        N.check(code, self._h, what)

    def status(self):
        self._check(self._lib.gna_plan_status(self._h), "gna_plan_status")

    def info(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.gna_plan_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "info")
        return {"nodes": a.value, "points_per_eval": b.value, "device_bytes": c.value}

    @property
    def launches(self) -> int:
        return self._lib.gna_plan_kernel_launches(self._h)

    @property
    def tuning(self) -> str:
        buf = ctypes.create_string_buffer(128)
        self._check(self._lib.gna_plan_get_tuning(self._h, buf, 128), "get_tuning")
        return buf.value.decode()

    @tuning.setter
    def tuning(self, text: str):
        self._check(self._lib.gna_plan_set_tuning(self._h, text.encode()), "set_tuning")

    def set_graph(self, on: bool):
        self._check(self._lib.gna_plan_set_graph(self._h, int(bool(on))), "set_graph")

    def profile(self, on):
        """Record CUDA events around the fused node kernel of every evaluation
        (on = True or 1), of every k-th one (on = k), or not (on = False or 0)."""
        self._check(self._lib.gna_plan_profile(self._h, int(on)), "profile")

    def profile_read(self):
        """(summed fused-kernel ms, timed launches) since the last read."""
        ms, n = ctypes.c_double(), ctypes.c_int()
        self._check(self._lib.gna_plan_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n)), "profile_read")
        return ms.value, n.value

    # ------------------------------------------ autograd Function's path --
    def _ad_check(self, theta, eta, data) -> int:
        """Arguments of OscChi2 on this plan (one point); returns the parameter count."""
        npar = 4 if self.channel is None else 6
        if self.npts != 1:
            raise ValueError("OscChi2 works on a single-point plan")
        ok = lambda t, n: (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                           and t.numel() == n and t.is_contiguous())
        if not ok(theta, npar):
            raise ValueError("theta must be a contiguous float64 CUDA tensor of %d values" % npar)
        if eta is not None and not ok(eta, self.nbins):
            raise ValueError("eta must be a contiguous float64 CUDA tensor of nbins values")
        if not ok(data, self.nbins):
            raise ValueError("data must be a contiguous float64 CUDA tensor of nbins values")
        return npar

    def _eval_into(self, p, data, e, sigma, chi2, g_theta, g_eta):
        """One evaluation writing chi2, d chi2 / d theta into g_theta and (with
        nuisances) d chi2 / d eta into g_eta, through a ctypes output struct
        kept by the plan."""
        o = self.__dict__.get("_ad_out")
        if o is None:
            o = self._ad_out = N.GnaOutputs()
        o.chi2, o.grad = chi2.data_ptr(), g_theta.data_ptr()
        o.grad_eta = None if g_eta is None else g_eta.data_ptr()
        fn = self._lib.gna_chain_eval if self.channel is None else self._lib.gna_chain_eval_general
        code = fn(self._h, p.data_ptr(), None if e is None else e.data_ptr(), float(sigma), data.data_ptr(), 0,
                  ctypes.byref(o), torch.cuda.current_stream().cuda_stream)
        if code != N.GNA_OK:
            self._check(code, "gna_chain_eval")

    # ------------------------------------------------------- evaluation --
    def params_tensor(self, theta) -> torch.Tensor:
        npar = 4 if self.channel is None else 6
        t = torch.as_tensor(np.asarray(theta, dtype=np.float64).reshape(-1, npar), device=self.device)
        if t.shape[0] != self.npts:
            raise ValueError("expected %d parameter points" % self.npts)
        return t.contiguous()

    def _out(self, name, shape):
        return torch.empty(shape, dtype=torch.float64, device=self.device)

    def eval(self, params: torch.Tensor, data: torch.Tensor, eta: Optional[torch.Tensor] = None, sigma: float = 0.0,
             grad: bool = True, grad_eta: bool = False, mu: bool = False, spectra: bool = False, plain: bool = False,
             out: Optional[dict] = None, stream=None) -> dict:
        """One evaluation of all points.  params [npts, 4] float64 CUDA; data [nbins] or [npts, nbins]."""
        if params.dtype != torch.float64 or tuple(params.shape) != (self.npts, 4):
            raise ValueError("params must be float64 [npts, 4]")
        dpp = 1 if data.dim() == 2 else 0
        if data.dtype != torch.float64 or data.shape[-1] != self.nbins or (dpp and data.shape[0] != self.npts):
            raise ValueError("data must be float64 [nbins] or [npts, nbins]")
        if eta is not None and (eta.dtype != torch.float64 or eta.numel() != self.nbins):
            raise ValueError("eta must be float64 [nbins]")
        if out is None:
            out = {"chi2": self._out("chi2", (self.npts,))}
            if grad:
                out["grad"] = self._out("grad", (self.npts, 4))
            if grad_eta:
                out["grad_eta"] = self._out("grad_eta", (self.npts, self.nbins))
            if mu:
                out["mu"] = self._out("mu", (self.npts, self.nbins))
            if spectra:
                out["spectra"] = self._out("spectra", (self.npts, self.nL, self.nbins))
        o = N.GnaOutputs(_ptr(out["chi2"]), _ptr(out.get("grad")), _ptr(out.get("grad_eta")), _ptr(out.get("mu")),
                         _ptr(out.get("spectra")))
        fn = self._lib.gna_chain_eval_plain if plain else self._lib.gna_chain_eval
        code = fn(self._h, _ptr(params), _ptr(eta), float(sigma), _ptr(data), dpp, ctypes.byref(o),
                  ctypes.c_void_p(_stream(stream)))
        self._check(code, "gna_chain_eval_plain" if plain else "gna_chain_eval")
        return out

    def eval_general(self, params: torch.Tensor, data: torch.Tensor, eta: Optional[torch.Tensor] = None,
                     sigma: float = 0.0, grad: bool = True, grad_eta: bool = False, mu: bool = False,
                     out: Optional[dict] = None, stream=None) -> dict:
        """One evaluation of all points of an any-channel plan.  params [npts, 6]
        float64 CUDA (s2_12, s2_13, s2_23, delta_cp, dm2_21, dm2_32); data [nbins]
        or [npts, nbins]; out["grad"] is [npts, 6]."""
        if self.channel is None:
            raise ValueError("the plan was created without a channel")
        if params.dtype != torch.float64 or tuple(params.shape) != (self.npts, 6):
            raise ValueError("params must be float64 [npts, 6]")
        dpp = 1 if data.dim() == 2 else 0
        if data.dtype != torch.float64 or data.shape[-1] != self.nbins or (dpp and data.shape[0] != self.npts):
            raise ValueError("data must be float64 [nbins] or [npts, nbins]")
        if eta is not None and (eta.dtype != torch.float64 or eta.numel() != self.nbins):
            raise ValueError("eta must be float64 [nbins]")
        if out is None:
            out = {"chi2": self._out("chi2", (self.npts,))}
            if grad:
                out["grad"] = self._out("grad6", (self.npts, 6))
            if grad_eta:
                out["grad_eta"] = self._out("grad_eta", (self.npts, self.nbins))
            if mu:
                out["mu"] = self._out("mu", (self.npts, self.nbins))
        o = N.GnaOutputs(_ptr(out["chi2"]), _ptr(out.get("grad")), _ptr(out.get("grad_eta")), _ptr(out.get("mu")),
                         None)
        code = self._lib.gna_chain_eval_general(self._h, _ptr(params), _ptr(eta), float(sigma), _ptr(data), dpp,
                                                ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
        self._check(code, "gna_chain_eval_general")
        return out

    def eval_cached(self, data: torch.Tensor, eta: Optional[torch.Tensor] = None, sigma: float = 0.0,
                    grad: bool = True, grad_eta: bool = False, mu: bool = False, spectra: bool = False,
                    out: Optional[dict] = None, stream=None) -> dict:
        """The epilogue only (nuisances, chi^2, gradient) on the node sums the last
        evaluation kept: new eta / data, the same oscillation parameters."""
        dpp = 1 if data.dim() == 2 else 0
        if data.dtype != torch.float64 or data.shape[-1] != self.nbins or (dpp and data.shape[0] != self.npts):
            raise ValueError("data must be float64 [nbins] or [npts, nbins]")
        if out is None:
            out = {"chi2": self._out("chi2", (self.npts,))}
            if grad:
                out["grad"] = self._out("grad", (self.npts, 4))
            if grad_eta:
                out["grad_eta"] = self._out("grad_eta", (self.npts, self.nbins))
            if mu:
                out["mu"] = self._out("mu", (self.npts, self.nbins))
            if spectra:
                out["spectra"] = self._out("spectra", (self.npts, self.nL, self.nbins))
        o = N.GnaOutputs(_ptr(out["chi2"]), _ptr(out.get("grad")), _ptr(out.get("grad_eta")), _ptr(out.get("mu")),
                         _ptr(out.get("spectra")))
        code = self._lib.gna_chain_eval_cached(self._h, _ptr(eta), float(sigma), _ptr(data), dpp, ctypes.byref(o),
                                               ctypes.c_void_p(_stream(stream)))
        self._check(code, "gna_chain_eval_cached")
        return out

    def eval_host(self, params: np.ndarray, data: np.ndarray, eta: Optional[np.ndarray] = None, sigma: float = 0.0,
                  grad: bool = True, chi2_out: Optional[np.ndarray] = None, grad_out: Optional[np.ndarray] = None,
                  spectra_out: Optional[np.ndarray] = None, stream=None):
        """Evaluation from host buffers (copies in, evaluates, copies out,
        synchronises).  params [npts, 4], or [npts, 6] on an any-channel plan
        (which has no spectra)."""
        npar = self._npar
        p = np.ascontiguousarray(params, dtype=np.float64).reshape(self.npts, npar)
        d = np.ascontiguousarray(data, dtype=np.float64)
        e = None if eta is None else np.ascontiguousarray(eta, dtype=np.float64)
        dpp = 1 if d.ndim == 2 else 0
        c = chi2_out if chi2_out is not None else np.empty(self.npts)
        g = (grad_out if grad_out is not None else np.empty((self.npts, npar))) if grad else None
        vp = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
        if self.channel is not None:
            if spectra_out is not None:
                raise ValueError("the any-channel chain has no per-baseline spectra")
            code = self._lib.gna_chain_eval_general_host(self._h, vp(p), vp(e), float(sigma), vp(d), dpp, vp(c), vp(g),
                                                         ctypes.c_void_p(_stream(stream)))
            self._check(code, "gna_chain_eval_general_host")
            return c, g
        code = self._lib.gna_chain_eval_host(self._h, vp(p), vp(e), float(sigma), vp(d), dpp, vp(c), vp(g),
                                             vp(spectra_out), ctypes.c_void_p(_stream(stream)))
        self._check(code, "gna_chain_eval_host")
        return c, g

    @property
    def _npar(self) -> int:
        return 4 if self.channel is None else 6

    def eval_host_async(self, params: np.ndarray, data: np.ndarray, eta: Optional[np.ndarray] = None,
                        sigma: float = 0.0, grad: bool = True, spectra: bool = False, stream=None) -> int:
        """Enqueues an evaluation from host buffers and returns a ticket at once
        (at most two outstanding); eval_host_wait(ticket) takes its results."""
        p = np.ascontiguousarray(params, dtype=np.float64).reshape(self.npts, self._npar)
        d = np.ascontiguousarray(data, dtype=np.float64)
        e = None if eta is None else np.ascontiguousarray(eta, dtype=np.float64)
        dpp = 1 if d.ndim == 2 else 0
        vp = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
        t = ctypes.c_int64(-1)
        if self.channel is not None:
            if spectra:
                raise ValueError("the any-channel chain has no per-baseline spectra")
            code = self._lib.gna_chain_eval_general_host_async(self._h, vp(p), vp(e), float(sigma), vp(d), dpp,
                                                               int(bool(grad)), ctypes.c_void_p(_stream(stream)),
                                                               ctypes.byref(t))
            self._check(code, "gna_chain_eval_general_host_async")
            return t.value
        code = self._lib.gna_chain_eval_host_async(self._h, vp(p), vp(e), float(sigma), vp(d), dpp, int(bool(grad)),
                                                   int(bool(spectra)), ctypes.c_void_p(_stream(stream)), ctypes.byref(t))
        self._check(code, "gna_chain_eval_host_async")
        return t.value

    def eval_host_wait(self, ticket: int, chi2_out: Optional[np.ndarray] = None, grad_out: Optional[np.ndarray] = None,
                       spectra_out: Optional[np.ndarray] = None):
        """Waits for the evaluation `ticket` and unpacks (chi2, grad) and, if given, the spectra."""
        c = chi2_out if chi2_out is not None else np.empty(self.npts)
        g = grad_out if grad_out is not None else np.empty((self.npts, self._npar))
        vp = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
        code = self._lib.gna_chain_eval_host_wait(self._h, ctypes.c_int64(ticket), vp(c), vp(g), vp(spectra_out))
        self._check(code, "gna_chain_eval_host_wait")
        return c, g

    def fit(self, params: torch.Tensor, data: torch.Tensor, iters: int = 20, lambda0: float = 1e-3,
            graph: bool = True, chi2_out: Optional[torch.Tensor] = None, stream=None):
        """Batched Levenberg-Marquardt fits; params [npts, 4] ([npts, 6] on an
        any-channel plan) float64 CUDA is overwritten with the best points."""
        npar = self._npar
        if params.dtype != torch.float64 or tuple(params.shape) != (self.npts, npar) or not params.is_contiguous():
            raise ValueError("params must be a contiguous float64 tensor [npts, %d]" % npar)
        if data.dtype != torch.float64 or tuple(data.shape) != (self.npts, self.nbins):
            raise ValueError("data must be float64 [npts, nbins]")
        if chi2_out is None:
            chi2_out = self._out("fit_chi2", (self.npts,))
        fn, what = ((self._lib.gna_fit_batch, "gna_fit_batch") if self.channel is None else
                    (self._lib.gna_fit_batch_general, "gna_fit_batch_general"))
        code = fn(self._h, _ptr(params), _ptr(data), int(iters), float(lambda0), _ptr(chi2_out), int(bool(graph)),
                  ctypes.c_void_p(_stream(stream)))
        self._check(code, what)
        return params, chi2_out

    def autotune(self, params: torch.Tensor, data: torch.Tensor, reps: int = 3, grad: bool = True,
                 mu: bool = False, spectra: bool = False, stream=None) -> str:
        """Times the candidate mappings and launch shapes with the outputs the
        caller will ask for (the kernels differ with them) and keeps the fastest."""
        dpp = 1 if data.dim() == 2 else 0
        out = {"chi2": self._out("chi2", (self.npts,))}
        if grad:
            out["grad"] = self._out("grad", (self.npts, 4 if self.channel is None else 6))
        if mu:
            out["mu"] = self._out("mu", (self.npts, self.nbins))
        if self.channel is not None:
            o = N.GnaOutputs(_ptr(out["chi2"]), _ptr(out.get("grad")), None, _ptr(out.get("mu")), None)
            code = self._lib.gna_plan_autotune_general(self._h, _ptr(params), _ptr(data), dpp, ctypes.byref(o),
                                                       int(reps), ctypes.c_void_p(_stream(stream)))
            self._check(code, "gna_plan_autotune_general")
            return self.tuning
        if spectra:
            out["spectra"] = self._out("spectra", (self.npts, self.nL, self.nbins))
        o = N.GnaOutputs(_ptr(out["chi2"]), _ptr(out.get("grad")), None, _ptr(out.get("mu")), _ptr(out.get("spectra")))
        code = self._lib.gna_plan_autotune(self._h, _ptr(params), _ptr(data), dpp, ctypes.byref(o), int(reps),
                                           ctypes.c_void_p(_stream(stream)))
        self._check(code, "gna_plan_autotune")
        return self.tuning


def _check_noalloc_args(E, W, Ls, Lw, params, data, out):
    """Refuses, before anything reaches the library, every argument of
    chi2_noalloc whose dtype, shape or device would make the kernels read or
    write outside the caller's buffers: dtypes and shapes first, then that all
    tensors are contiguous CUDA tensors on E's device."""
    f64 = torch.float64
    if not isinstance(E, torch.Tensor) or E.dtype != f64 or E.dim() != 2:
        raise ValueError("E must be a float64 tensor [nbins, n]")
    nbins = E.shape[0]
    if not isinstance(W, torch.Tensor) or W.dtype != f64 or tuple(W.shape) != tuple(E.shape):
        raise ValueError("W must be a float64 tensor shaped like E %s" % (tuple(E.shape),))
    if not isinstance(params, torch.Tensor) or params.dtype != f64 or params.numel() != 4:
        raise ValueError("params must be a float64 tensor of 4 values [1, 4]")
    if not isinstance(data, torch.Tensor) or data.dtype != f64 or data.numel() != nbins:
        raise ValueError("data must be a float64 tensor of nbins = %d values" % nbins)
    if Ls.ndim != 1 or Ls.size < 1 or (Lw is not None and Lw.shape != Ls.shape):
        raise ValueError("L must hold one or more baselines and Lweight (if given) one weight per baseline")
    tensors = [E, W, params, data]
    if out is not None:
        need = {"chi2": 1, "grad": 4, "mu": nbins}
        if "chi2" not in out:
            raise ValueError("out must hold 'chi2'")
        for k, t in out.items():
            if k not in need:
                raise ValueError("unknown output %r" % k)
            if not isinstance(t, torch.Tensor) or t.dtype != f64 or t.numel() < need[k]:
                raise ValueError("out[%r] must be a float64 tensor of at least %d values" % (k, need[k]))
            tensors.append(t)
    for t in tensors:
        if not t.is_cuda or t.device != E.device:
            raise ValueError("all tensors must be CUDA tensors on E's device")
        if not t.is_contiguous():
            raise ValueError("all tensors must be contiguous")


def chi2_noalloc(E: torch.Tensor, W: torch.Tensor, L, params: torch.Tensor, data: torch.Tensor, norm: float,
                 kind="pearson", Lweight=None, grad: bool = True, mu: bool = False, out: Optional[dict] = None,
                 stream=None) -> dict:
    """chi^2 of one point without any device allocation in the library.

    For callers that cannot allocate device memory (a pool or arena they do not
    own, a host framework that forbids cudaMalloc): the library works in a
    fixed ~0.9 MB array of its own, shared by all calls, so calls must not
    overlap on the GPU.  E, W: [nbins, n] float64 (node energies in MeV, node
    weights); params [1, 4]; data [nbins].  Output tensors may be passed in
    ``out`` (chi2 [1], grad [4], mu [nbins]) so that this call allocates
    nothing on the Python side either.
    """
    Ls = _f64(np.atleast_1d(L))
    Lw = None if Lweight is None else _f64(Lweight)
    _check_noalloc_args(E, W, Ls, Lw, params, data, out)
    _require_cuda()
    nbins, n = E.shape
    if out is None:
        out = {"chi2": torch.empty(1, dtype=torch.float64, device=E.device)}
        if grad:
            out["grad"] = torch.empty(4, dtype=torch.float64, device=E.device)
        if mu:
            out["mu"] = torch.empty(nbins, dtype=torch.float64, device=E.device)
    P = ctypes.POINTER(ctypes.c_double)
    code = N.lib().gna_chain_eval_noalloc(int(nbins), int(n), _ptr(E), _ptr(W), Ls.ctypes.data_as(P), Ls.size,
                                          None if Lw is None else Lw.ctypes.data_as(P), _ptr(params), float(norm),
                                          KINDS[kind], _ptr(data), _ptr(out["chi2"]), _ptr(out.get("grad")),
                                          _ptr(out.get("mu")), ctypes.c_void_p(_stream(stream)))
    N.check(code, what="gna_chain_eval_noalloc")
    return out


class OscChi2(torch.autograd.Function):
    """chi^2(theta, eta) of one plan point with its hand-written gradient.

    theta has 4 parameters on a survival-chain plan and 6 on an any-channel
    plan.  forward runs one fused evaluation with the tangents on and keeps
    d chi2 / d theta (and d chi2 / d eta); backward scales the kept gradient
    by grad_output in place (one launch) and returns it, so one chi2 can be
    differentiated once (a second backward through it raises RuntimeError).
    """

    @staticmethod
    def forward(ctx, theta, eta, plan: Plan, data, sigma: float = 0.0):
        npar = plan._ad_check(theta, eta, data)
        # the library writes chi2 and the gradient straight into the tensors
        # this call returns and keeps (no copies); only pointers are read
        # in the inputs' shapes, so that no view is needed; kept on ctx (an
        # intermediate of this call: no saved-tensor bookkeeping)
        chi2 = torch.empty((), dtype=torch.float64, device=theta.device)
        ctx.g_theta = torch.empty(theta.shape, dtype=torch.float64, device=theta.device)
        ctx.g_eta = None if eta is None else torch.empty(eta.shape, dtype=torch.float64, device=theta.device)
        plan._eval_into(theta, data, eta, sigma, chi2, ctx.g_theta, ctx.g_eta)
        ctx.lib = plan._lib
        return chi2

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, go):
        # the kept gradient is scaled by grad_output in place, one launch for
        # theta and eta (gna_grad_scale), and handed to the gradient
        # accumulation, which takes fresh non-view tensors as they are; so
        # it can be handed out once
        if ctx.g_theta is None:
            raise RuntimeError("OscChi2: a second backward through the same chi2 needs a new evaluation")
        gt, ge = ctx.g_theta, ctx.g_eta
        ctx.g_theta = ctx.g_eta = None
        if not (go.is_cuda and go.dtype == torch.float64 and go.device == gt.device and go.numel() == 1):
            raise ValueError("OscChi2: grad_output must be a float64 scalar on the evaluation's device")
        code = ctx.lib.gna_grad_scale(gt.data_ptr(), gt.numel(), None if ge is None else ge.data_ptr(),
                                      0 if ge is None else ge.numel(), go.data_ptr(),
                                      torch.cuda.current_stream(gt.device).cuda_stream)
        N.check(code, what="gna_grad_scale")
        return gt, ge, None, None, None


def chi2(theta, plan: Plan, data, eta=None, sigma: float = 0.0):
    return OscChi2.apply(theta, eta, plan, data, sigma)
