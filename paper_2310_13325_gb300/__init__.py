"""GB300-native hot path of variational Bayesian full-waveform inversion.

Thin Python layer over libvipgb (include/vipgb.h): argument checking and
marshalling of torch CUDA tensors into the C ABI. Every step of the
computation runs in the library's CUDA kernels; there is no CPU fallback -
calls fail loudly when the library is missing or a tensor is not on a GPU.

Entry points follow the paper (Zhang & Curtis, arXiv 2310.13325):
  Fwi.forward / Fwi.gradient / Fwi.adjoint   wave simulation, Gaussian misfit
                                             (Eq. 26), adjoint-state gradient
  FwiSeis                                    torch.autograd.Function of the
                                             seismogram map
  svgd_step (Eq. 17), ssvgd_step (Eq. 22, 25), advi_sample / advi_step
  (Eq. 10-12, mean-field), philox_normal
  Tomo.traveltimes / Tomo.gradient          travel-time tomography (Sec. 4.1):
                                             eikonal travel times, ray gradient
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import FwiGeom, VipError, check

FWI_FP32, FWI_CKPT_BF16, FWI_CKPT_FP16 = 0, 1, 2
VIP_OK, VIP_ERR_ARG, VIP_ERR_CFL, VIP_ERR_NOMEM, VIP_ERR_CUDA = 0, -1, -2, -3, -4
VIP_ERR_TIMEOUT, VIP_ERR_NOTPD, VIP_ERR_UNSUPPORTED, VIP_ERR_NONFINITE = -5, -6, -7, -8
FWI_MODE_BATCHED, FWI_MODE_PLAIN = 0, 1
VIP_GRAM_BF16, VIP_GRAM_BF16X3, VIP_GRAM_FP32 = 0, 1, 2

__all__ = ["Fwi", "FwiSeis", "Tomo", "svgd_step", "ssvgd_step", "svgd_inverse_variance",
           "advi_step_opt", "advi_lowrank_sample", "advi_lowrank_step", "to_unconstrained", "to_model", "unconstrained_gradient",
           "ASCENT_SGD", "ASCENT_ADAGRAD", "ASCENT_ADADELTA", "ASCENT_ADAM", "advi_sample", "advi_step",
           "philox_normal", "svgd_workspace_size", "svgd_sqdist", "svgd_step_noalloc", "FWI_FP32", "FWI_CKPT_BF16",
           "FWI_CKPT_FP16", "FWI_MODE_BATCHED", "FWI_MODE_PLAIN", "VIP_GRAM_BF16",
           "VIP_GRAM_BF16X3", "VIP_GRAM_FP32", "VipError", "svgd_status", "VIP_OK",
           "VIP_ERR_ARG", "VIP_ERR_CFL", "VIP_ERR_NOMEM", "VIP_ERR_CUDA", "VIP_ERR_TIMEOUT",
           "VIP_ERR_NOTPD", "VIP_ERR_UNSUPPORTED", "VIP_ERR_NONFINITE"]


def _torch():
    import torch
    return torch


def _ptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (or None -> NULL)."""
    if t is None:
        return None
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Fwi:
    """FWI context for one acquisition geometry (wraps fwi_create)."""

    def __init__(self, nz, nx, dx, dt, nt, src_iz, src_ix, rec_iz, rec_ix, f0=10.0,
                 t0=0.0, nsponge=20, sponge_alpha=0.015, workspace_limit=0):
        L = _lib.load()
        self.nz, self.nx, self.nt = int(nz), int(nx), int(nt)
        self._arrays = [np.ascontiguousarray(a, dtype=np.int32)
                        for a in (src_iz, src_ix, rec_iz, rec_ix)]
        self.S = self._arrays[0].size
        self.R = self._arrays[2].size
        cp = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) for a in self._arrays]
        g = FwiGeom(self.nz, self.nx, float(dx), float(dt), self.nt, int(nsponge),
                    float(sponge_alpha), float(f0), float(t0), self.S, cp[0], cp[1],
                    self.R, cp[2], cp[3])
        h = ctypes.c_void_p()
        check(L.fwi_create(ctypes.byref(g), int(workspace_limit), ctypes.byref(h)),
              "fwi_create")
        self._h = h
        self._L = L

    @classmethod
    def from_config(cls, cfg, geo, **kw):
        return cls(cfg.nz, cfg.nx, cfg.dx, cfg.dt, cfg.nt, geo["src_iz"], geo["src_ix"],
                   geo["rec_iz"], geo["rec_ix"], f0=cfg.f0, nsponge=cfg.nsponge,
                   sponge_alpha=cfg.sponge_alpha, **kw)

    def close(self):
        if getattr(self, "_h", None):
            self._L.fwi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mode(self, mode=FWI_MODE_BATCHED, ckpt_every=1):
        check(self._L.fwi_set_mode(self._h, int(mode), int(ckpt_every)), "fwi_set_mode")

    def set_plan(self, Q=0, V=0, T=0, sources_per_item=0, coeff=0):
        """Force the batched launch shape (cluster CTAs, rows per thread,
        threads per CTA, sources per work item, coefficients in shared (1) or
        global (2) memory); zeros = automatic."""
        check(self._L.fwi_set_plan(self._h, int(Q), int(V), int(T), int(sources_per_item),
                                   int(coeff)), "fwi_set_plan")

    def set_autotune(self, enable=True):
        check(self._L.fwi_set_autotune(self._h, int(bool(enable))), "fwi_set_autotune")

    def set_fill(self, enable=True):
        """Enable or disable the second launch on the SMs the batched launch
        leaves idle (fwi_set_fill)."""
        check(self._L.fwi_set_fill(self._h, int(bool(enable))), "fwi_set_fill")

    def query_fill(self, P, precision=FWI_FP32):
        """Shape of the fill launch a gradient call for P particles would add
        (all zeros: none)."""
        out = (ctypes.c_int * 4)()
        check(self._L.fwi_query_fill(self._h, int(P), int(precision), out), "fwi_query_fill")
        return dict(zip(("cluster_ctas", "rows_per_thread", "threads", "clusters"), list(out)))

    def query_plan(self, P, precision=FWI_FP32):
        out = (ctypes.c_int * 10)()
        nb = ctypes.c_size_t()
        check(self._L.fwi_query_plan(self._h, int(P), int(precision), out,
                                     ctypes.byref(nb)), "fwi_query_plan")
        keys = ("cluster_ctas", "rows_per_thread", "threads", "band_rows",
                "concurrent_pairs", "ckpt_every", "work_items", "sources_per_item")
        d = dict(zip(keys, list(out)))
        d["coefficients"] = "global" if out[8] == 2 else "shared"
        d["smem_bytes"] = out[9]
        d["scratch_bytes"] = nb.value
        return d

    def last_status(self):
        return self._L.fwi_last_status(self._h)

    def bytes_needed(self):
        """Device scratch bytes the last planned call needed (or, after
        VIP_ERR_NOMEM, the smallest footprint it could not fit)."""
        return int(self._L.fwi_bytes_needed(self._h))

    def _models(self, v):
        """Accept one model [nz, nx] or a batch [P, nz, nx] / [P, nz*nx]."""
        d = self.nz * self.nx
        if tuple(v.shape) == (self.nz, self.nx) or (v.dim() == 1 and v.numel() == d):
            v = v.reshape(1, d)
        elif v.dim() == 3 and tuple(v.shape[1:]) == (self.nz, self.nx):
            pass
        elif v.dim() == 2 and v.shape[1] == d:
            pass
        else:
            raise ValueError("models must be [nz, nx], [P, nz, nx] or [P, nz*nx]")
        return v.reshape(v.shape[0], self.nz, self.nx).contiguous(), v.shape[0]

    def forward(self, v, out=None, stream=None):
        torch = _torch()
        v, P = self._models(v)
        if out is None:
            out = torch.empty((P, self.S, self.R, self.nt), device=v.device,
                              dtype=torch.float32)
        check(self._L.fwi_forward(self._h, _ptr(v, torch.float32, "v"), P,
                                  _ptr(out, torch.float32, "seis"), _stream(stream)),
              "fwi_forward")
        return out

    def gradient(self, v, dobs, sigma, precision=FWI_FP32, misfit=None, grad=None,
                 stream=None, sources=None):
        """Returns (misfit [P] float64, dJ/dv [P, nz, nx]). With sources (a
        sequence of distinct source indices) both are sums over that minibatch
        of sources only (fwi_gradient_sources)."""
        torch = _torch()
        v, P = self._models(v)
        if misfit is None:
            misfit = torch.empty(P, device=v.device, dtype=torch.float64)
        if grad is None:
            grad = torch.empty((P, self.nz, self.nx), device=v.device, dtype=torch.float32)
        if tuple(dobs.shape) != (self.S, self.R, self.nt):
            raise ValueError("dobs must be [S, R, nt]")
        if sources is None:
            check(self._L.fwi_gradient(self._h, _ptr(v, torch.float32, "v"), P,
                                       _ptr(dobs, torch.float32, "dobs"), float(sigma),
                                       _ptr(misfit, torch.float64, "misfit"),
                                       _ptr(grad, torch.float32, "grad"), int(precision),
                                       _stream(stream)), "fwi_gradient")
        else:
            src = [int(s) for s in sources]
            arr = (ctypes.c_int * len(src))(*src)
            check(self._L.fwi_gradient_sources(self._h, _ptr(v, torch.float32, "v"), P,
                                               _ptr(dobs, torch.float32, "dobs"), float(sigma),
                                               ctypes.cast(arr, ctypes.c_void_p), len(src),
                                               _ptr(misfit, torch.float64, "misfit"),
                                               _ptr(grad, torch.float32, "grad"),
                                               int(precision), _stream(stream)),
                  "fwi_gradient_sources")
        return misfit, grad

    def adjoint(self, v, dseis, precision=FWI_FP32, grad=None, stream=None):
        torch = _torch()
        v, P = self._models(v)
        if grad is None:
            grad = torch.empty((P, self.nz, self.nx), device=v.device, dtype=torch.float32)
        if tuple(dseis.shape) != (P, self.S, self.R, self.nt):
            raise ValueError("dseis must be [P, S, R, nt]")
        check(self._L.fwi_adjoint(self._h, _ptr(v, torch.float32, "v"), P,
                                  _ptr(dseis.contiguous(), torch.float32, "dseis"),
                                  _ptr(grad, torch.float32, "grad"), int(precision),
                                  _stream(stream)), "fwi_adjoint")
        return grad


class Tomo:
    """Travel-time tomography context (wraps tomo_create): ny x nx nodes of
    spacing h km, stations as node indices i * nx + j (Sec. 4.1)."""

    def __init__(self, ny, nx, h, stations):
        L = _lib.load()
        self.ny, self.nx, self.h = int(ny), int(nx), float(h)
        self._sta = np.ascontiguousarray(stations, dtype=np.int32)
        self.ns = self._sta.size
        h_ = ctypes.c_void_p()
        check(L.tomo_create(self.ny, self.nx, self.h, self.ns,
                            self._sta.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            ctypes.byref(h_)), "tomo_create")
        self._h = h_
        self._L = L
        self.n_pairs = L.tomo_pair_count(h_)

    @classmethod
    def from_config(cls, cfg, stations):
        return cls(cfg.ny, cfg.nx, cfg.h, stations)

    def close(self):
        if getattr(self, "_h", None):
            self._L.tomo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_status(self):
        return self._L.tomo_last_status(self._h)

    def _models(self, V):
        d = self.ny * self.nx
        if V.dim() == 1 and V.numel() == d or tuple(V.shape) == (self.ny, self.nx):
            V = V.reshape(1, d)
        elif not ((V.dim() == 2 and V.shape[1] == d) or
                  (V.dim() == 3 and tuple(V.shape[1:]) == (self.ny, self.nx))):
            raise ValueError("velocity maps must be [P, ny, nx] or [P, ny*nx]")
        return V, int(V.shape[0])

    def traveltimes(self, V, out=None, stream=None):
        """Travel times [P, n_pairs] (s) of the station pairs, s-major."""
        torch = _torch()
        V, P = self._models(V)
        if out is None:
            out = torch.empty((P, self.n_pairs), device=V.device, dtype=torch.float32)
        check(self._L.tomo_traveltimes(self._h, _ptr(V, torch.float32, "V"), P,
                                       _ptr(out, torch.float32, "out"), _stream(stream)),
              "tomo_traveltimes")
        return out

    def gradient(self, V, dobs, sigma, misfit=None, grad=None, T=None, sources=None,
                 stream=None):
        """Misfit [P] (FP64) and dJ/dv [P, ny, nx] from rays (Eq. 26); sources
        (host list of source stations) sums only their pairs (a minibatch)."""
        torch = _torch()
        V, P = self._models(V)
        if misfit is None:
            misfit = torch.empty(P, device=V.device, dtype=torch.float64)
        if grad is None:
            grad = torch.empty((P, self.ny, self.nx), device=V.device, dtype=torch.float32)
        for name, t in (("dobs", dobs), ("sigma", sigma)):
            if t.numel() != self.n_pairs:
                raise ValueError("%s must hold %d travel times" % (name, self.n_pairs))
        if sources is not None:
            if T is not None:
                raise ValueError("T is not reported for a source minibatch")
            src = [int(k) for k in sources]
            arr = (ctypes.c_int * len(src))(*src)
            check(self._L.tomo_gradient_sources(self._h, _ptr(V, torch.float32, "V"), P,
                                                _ptr(dobs, torch.float32, "dobs"),
                                                _ptr(sigma, torch.float32, "sigma"),
                                                ctypes.cast(arr, ctypes.c_void_p), len(src),
                                                _ptr(misfit, torch.float64, "misfit"),
                                                _ptr(grad, torch.float32, "grad"),
                                                _stream(stream)), "tomo_gradient_sources")
            return misfit, grad
        check(self._L.tomo_gradient(self._h, _ptr(V, torch.float32, "V"), P,
                                    _ptr(dobs, torch.float32, "dobs"),
                                    _ptr(sigma, torch.float32, "sigma"),
                                    _ptr(misfit, torch.float64, "misfit"),
                                    _ptr(grad, torch.float32, "grad"),
                                    _ptr(T, torch.float32, "T"), _stream(stream)),
              "tomo_gradient")
        return misfit, grad


def _make_fwiseis():
    torch = _torch()

    class FwiSeis(torch.autograd.Function):
        """Seismograms as a differentiable function of the velocity models:
        forward = fwi_forward, backward = fwi_adjoint (exact discrete adjoint)."""

        @staticmethod
        def forward(ctx, v, fwi):
            ctx.fwi = fwi
            ctx.save_for_backward(v)
            return fwi.forward(v.detach())

        @staticmethod
        def backward(ctx, gseis):
            (v,) = ctx.saved_tensors
            g = ctx.fwi.adjoint(v.detach(), gseis.contiguous())
            return g.reshape(v.shape), None

    return FwiSeis


class _Lazy:
    _cls = None

    def __getattr__(self, name):
        if _Lazy._cls is None:
            _Lazy._cls = _make_fwiseis()
        return getattr(_Lazy._cls, name)


FwiSeis = _Lazy()


def svgd_workspace_size(n, d, gram_precision=VIP_GRAM_BF16X3, stochastic=False):
    return int(_lib.load().svgd_workspace_size(int(n), int(d), int(gram_precision),
                                               int(bool(stochastic))))


def _workspace(n, d, gram_precision, stochastic, ws, device):
    torch = _torch()
    need = svgd_workspace_size(n, d, gram_precision, stochastic)
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=device)
    return ws


def svgd_sqdist(X, gram_precision=VIP_GRAM_BF16X3, ws=None, stream=None):
    """Squared pairwise distances D2 [n, n] (float64) of the particles X [n, d]
    and the median bandwidth h^2 (device float64 [1])."""
    torch = _torch()
    n, d = X.shape
    ws = _workspace(n, d, gram_precision, False, ws, X.device)
    D2 = torch.empty((n, n), dtype=torch.float64, device=X.device)
    h2 = torch.empty(1, dtype=torch.float64, device=X.device)
    check(_lib.load().svgd_sqdist(_ptr(X, torch.float32, "X"), n, d, int(gram_precision),
                                  _ptr(D2, torch.float64), _ptr(h2, torch.float64), _ptr(ws),
                                  ws.numel(), _stream(stream)), "svgd_sqdist")
    return D2, h2


def svgd_step(X, G, eps, h2=0.0, lo=None, hi=None, gram_precision=VIP_GRAM_BF16X3,
              ws=None, h2_used=None, gscale=1.0, q=None, stream=None):
    """In-place SVGD update of X [n, d] (Eq. 17) with grad log p = gscale * G;
    with q (device [d]) the diagonal matrix-valued kernel Q = diag(q)
    (svgd_step_q). Returns the workspace tensor (reusable) and h2_used
    (device float64 [1])."""
    torch = _torch()
    n, d = X.shape
    ws = _workspace(n, d, gram_precision, False, ws, X.device)
    if h2_used is None:
        h2_used = torch.empty(1, dtype=torch.float64, device=X.device)
    common = (n, d, float(eps), float(h2), _ptr(lo, torch.float32, "lo"),
              _ptr(hi, torch.float32, "hi"), int(gram_precision), _ptr(ws), ws.numel(),
              _ptr(h2_used, torch.float64), _stream(stream))
    if q is None:
        check(_lib.load().svgd_step(_ptr(X, torch.float32, "X"), _ptr(G, torch.float32, "G"),
                                    float(gscale), *common), "svgd_step")
    else:
        check(_lib.load().svgd_step_q(_ptr(X, torch.float32, "X"), _ptr(G, torch.float32, "G"),
                                      float(gscale), _ptr(q, torch.float32, "q"), *common),
              "svgd_step_q")
    return ws, h2_used


def svgd_status(ws, stream=None):
    """Status of the last SVGD call that used the workspace ws (synchronises
    the stream): VIP_OK, VIP_ERR_TIMEOUT or VIP_ERR_NONFINITE."""
    return int(_lib.load().svgd_status(_ptr(ws), _stream(stream)))


def svgd_inverse_variance(X, out=None, stream=None):
    """q [d] = 1 / variance of each coordinate across the particles X [n, d]
    (population variance; 1 where it is zero), the Q of the matrix-valued
    kernel."""
    torch = _torch()
    n, d = X.shape
    if out is None:
        out = torch.empty(d, dtype=torch.float32, device=X.device)
    check(_lib.load().svgd_inverse_variance(_ptr(X, torch.float32, "X"), n, d,
                                            _ptr(out, torch.float32, "q"), _stream(stream)),
          "svgd_inverse_variance")
    return out


def svgd_step_noalloc(X, G, eps, h2=0.0, lo=None, hi=None, gram_precision=VIP_GRAM_BF16X3,
                      h2_used=None, gscale=1.0, stream=None):
    """svgd_step whose scratch lives in the library's fixed device array
    (VIP_NOALLOC_SCRATCH_BYTES) instead of a caller workspace, for callers that
    cannot allocate device memory; no allocation happens inside the call.
    Overlapping calls on the GPU share that array and must not run at once."""
    torch = _torch()
    n, d = X.shape
    check(_lib.load().svgd_step_noalloc(_ptr(X, torch.float32, "X"),
                                        _ptr(G, torch.float32, "G"), float(gscale), n, d,
                                        float(eps), float(h2), _ptr(lo, torch.float32, "lo"),
                                        _ptr(hi, torch.float32, "hi"), int(gram_precision),
                                        _ptr(h2_used, torch.float64), _stream(stream)),
          "svgd_step_noalloc")


def ssvgd_step(X, G, eps, seed, it, xi=None, h2=0.0, lo=None, hi=None,
               gram_precision=VIP_GRAM_BF16X3, ws=None, h2_used=None, tau_used=None,
               gscale=1.0, q=None, stream=None):
    """In-place stochastic SVGD update of X [n, d] (Eq. 22 with the noise of
    Eq. 25); xi None draws the noise from Philox(seed, it) on the device; q
    (device [d]) selects the diagonal matrix-valued kernel (ssvgd_step_q)."""
    torch = _torch()
    n, d = X.shape
    ws = _workspace(n, d, gram_precision, True, ws, X.device)
    if h2_used is None:
        h2_used = torch.empty(1, dtype=torch.float64, device=X.device)
    if tau_used is None:
        tau_used = torch.empty(1, dtype=torch.float64, device=X.device)
    common = (n, d, float(eps), float(h2), _ptr(lo, torch.float32, "lo"),
              _ptr(hi, torch.float32, "hi"), int(gram_precision), _ptr(ws), ws.numel(),
              _ptr(h2_used, torch.float64), int(seed), int(it), _ptr(xi, torch.float32, "xi"),
              _ptr(tau_used, torch.float64), _stream(stream))
    if q is None:
        check(_lib.load().ssvgd_step(_ptr(X, torch.float32, "X"), _ptr(G, torch.float32, "G"),
                                     float(gscale), *common), "ssvgd_step")
    else:
        check(_lib.load().ssvgd_step_q(_ptr(X, torch.float32, "X"),
                                       _ptr(G, torch.float32, "G"), float(gscale),
                                       _ptr(q, torch.float32, "q"), *common), "ssvgd_step_q")
    return ws, h2_used, tau_used


def advi_sample(mu, omega, eta, a=None, b=None, out=None, stream=None):
    torch = _torch()
    S, d = eta.shape
    if out is None:
        out = torch.empty((S, d), dtype=torch.float32, device=mu.device)
    check(_lib.load().advi_sample(_ptr(mu, torch.float32, "mu"),
                                  _ptr(omega, torch.float32, "omega"),
                                  _ptr(eta, torch.float32, "eta"), S, d,
                                  _ptr(a, torch.float32, "a"), _ptr(b, torch.float32, "b"),
                                  _ptr(out, torch.float32, "m_out"), _stream(stream)),
          "advi_sample")
    return out


def advi_step(mu, omega, adam_state, t, eta, gm, lr, a=None, b=None, gscale=1.0, stream=None):
    """In-place Adam ascent of (mu, omega); adam_state [4, d] zero-initialised;
    d log p / dm = gscale * gm."""
    torch = _torch()
    S, d = eta.shape
    check(_lib.load().advi_step(_ptr(mu, torch.float32, "mu"),
                                _ptr(omega, torch.float32, "omega"),
                                _ptr(adam_state, torch.float32, "adam_state"), int(t),
                                _ptr(eta, torch.float32, "eta"), _ptr(gm, torch.float32, "gm"),
                                float(gscale), S, d, _ptr(a, torch.float32, "a"), _ptr(b, torch.float32, "b"),
                                float(lr), _stream(stream)), "advi_step")


ASCENT_SGD, ASCENT_ADAGRAD, ASCENT_ADADELTA, ASCENT_ADAM = 0, 1, 2, 3


def advi_step_opt(mu, omega, state, t, eta, gm, lr, rule, a=None, b=None, gscale=1.0,
                  stream=None):
    """advi_step with the ascent rule ASCENT_SGD, ASCENT_ADAGRAD,
    ASCENT_ADADELTA or ASCENT_ADAM; state [4, d] zero-initialised."""
    torch = _torch()
    S, d = eta.shape
    check(_lib.load().advi_step_opt(_ptr(mu, torch.float32, "mu"),
                                    _ptr(omega, torch.float32, "omega"),
                                    _ptr(state, torch.float32, "state"), int(t),
                                    _ptr(eta, torch.float32, "eta"),
                                    _ptr(gm, torch.float32, "gm"), float(gscale), S, d,
                                    _ptr(a, torch.float32, "a"), _ptr(b, torch.float32, "b"),
                                    float(lr), int(rule), _stream(stream)), "advi_step_opt")


def advi_lowrank_sample(mu, omega, B, eta, eps, a=None, b=None, out=None, stream=None):
    """m_s = T^{-1}(mu + e^omega eta_s + B eps_s); B [d, r], eta [S, d], eps [S, r]."""
    torch = _torch()
    S, d = eta.shape
    r = B.shape[1]
    if out is None:
        out = torch.empty((S, d), dtype=torch.float32, device=mu.device)
    check(_lib.load().advi_lowrank_sample(_ptr(mu, torch.float32, "mu"),
                                          _ptr(omega, torch.float32, "omega"),
                                          _ptr(B, torch.float32, "B"), r,
                                          _ptr(eta, torch.float32, "eta"),
                                          _ptr(eps, torch.float32, "eps"), S, d,
                                          _ptr(a, torch.float32, "a"), _ptr(b, torch.float32, "b"),
                                          _ptr(out, torch.float32, "m"), _stream(stream)),
          "advi_lowrank_sample")
    return out


def advi_lowrank_step(mu, omega, B, state, t, eta, eps, gm, lr, a=None, b=None, gscale=1.0,
                      work=None, stream=None):
    """In-place Adam ascent of (mu, omega, B) for Sigma = diag(e^{2 omega}) + B B^T;
    state [4 d + 2 d r] zero-initialised. Returns the FP64 work buffer (reusable)."""
    torch = _torch()
    S, d = eta.shape
    r = B.shape[1]
    if work is None:
        work = torch.empty(2 * r * r, dtype=torch.float64, device=mu.device)
    check(_lib.load().advi_lowrank_step(_ptr(mu, torch.float32, "mu"),
                                        _ptr(omega, torch.float32, "omega"),
                                        _ptr(B, torch.float32, "B"), r,
                                        _ptr(state, torch.float32, "state"),
                                        _ptr(work, torch.float64, "work"), int(t),
                                        _ptr(eta, torch.float32, "eta"),
                                        _ptr(eps, torch.float32, "eps"),
                                        _ptr(gm, torch.float32, "gm"), float(gscale), S, d,
                                        _ptr(a, torch.float32, "a"), _ptr(b, torch.float32, "b"),
                                        float(lr), _stream(stream)), "advi_lowrank_step")
    return work


def to_unconstrained(m, a, b, out=None, stream=None):
    """theta = log(m - a) - log(b - m) (Eq. 12), m [n, d], a, b [d]."""
    torch = _torch()
    n, d = m.shape
    out = torch.empty_like(m) if out is None else out
    check(_lib.load().vip_to_unconstrained(_ptr(m, torch.float32, "m"), _ptr(a, torch.float32, "a"),
                                           _ptr(b, torch.float32, "b"), n, d,
                                           _ptr(out, torch.float32, "theta"), _stream(stream)),
          "vip_to_unconstrained")
    return out


def to_model(theta, a, b, out=None, stream=None):
    """m = a + (b - a) / (1 + e^-theta) (Eq. 12)."""
    torch = _torch()
    n, d = theta.shape
    out = torch.empty_like(theta) if out is None else out
    check(_lib.load().vip_to_model(_ptr(theta, torch.float32, "theta"),
                                   _ptr(a, torch.float32, "a"), _ptr(b, torch.float32, "b"),
                                   n, d, _ptr(out, torch.float32, "m"), _stream(stream)),
          "vip_to_model")
    return out


def unconstrained_gradient(theta, gm, a, b, gscale=1.0, out=None, stream=None):
    """Gradient of the transformed log-density for theta from gscale * gm,
    the gradient in the model space at m = T^{-1}(theta)."""
    torch = _torch()
    n, d = theta.shape
    out = torch.empty_like(theta) if out is None else out
    check(_lib.load().vip_unconstrained_gradient(_ptr(theta, torch.float32, "theta"),
                                                 _ptr(gm, torch.float32, "gm"), float(gscale),
                                                 _ptr(a, torch.float32, "a"),
                                                 _ptr(b, torch.float32, "b"), n, d,
                                                 _ptr(out, torch.float32, "g"), _stream(stream)),
          "vip_unconstrained_gradient")
    return out


def philox_normal(rows, cols, seed, it, out=None, device="cuda"):
    torch = _torch()
    if out is None:
        out = torch.empty((rows, cols), dtype=torch.float32, device=device)
    check(_lib.load().vip_philox_normal(_ptr(out, torch.float32, "out"), int(rows),
                                        int(cols), int(seed), int(it), _stream()),
          "vip_philox_normal")
    return out
