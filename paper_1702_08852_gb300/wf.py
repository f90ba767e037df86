"""Python binding of the C ABI in include/wf.h (libwf.so).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  PyTorch supplies device memory and the CUDA stream.  The
functions carry the names of the C entry points (wf_plan, wf_solve, ...);
``Plan`` wraps a plan handle with the same calls as methods.

Tensors: maps are float64 CUDA tensors of length Npix (HEALPix RING order);
harmonic coefficients are complex128 CUDA tensors of length Nalm in m-major
order (index m (2 lmax + 1 - m) / 2 + l); masks are uint8/bool CUDA tensors.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libwf.so")

WF_OK, WF_ERR_ARG, WF_ERR_CUDA, WF_ERR_NOT_CONVERGED = 0, 1, 2, 3
WF_ERR_NUMERIC, WF_ERR_TIMEOUT, WF_ERR_UNIMPLEMENTED, WF_ERR_STATE = 4, 5, 6, 7
WF_PREC_FP64, WF_PREC_MIXED = 0, 1
WF_METHOD_DUAL, WF_METHOD_MESSENGER = 0, 1
WF_PCG_STOP_CAUCHY, WF_PCG_STOP_RESIDUAL = 0, 1
WF_STOP_CAUCHY, WF_STOP_ERROR = 0, 1


class WFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class wf_opts(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("eps_final", ctypes.c_double),
                ("eps_cap", ctypes.c_double), ("mu0", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("stop_rule", ctypes.c_int),
                ("precision", ctypes.c_int), ("band_limit", ctypes.c_int),
                ("graph_chunk", ctypes.c_int), ("refine_max", ctypes.c_int),
                ("timing", ctypes.c_int), ("autotune", ctypes.c_int),
                ("anchor", ctypes.c_int), ("anchor_eps", ctypes.c_double),
                ("anchor_cap", ctypes.c_double), ("anchor_cap_tol", ctypes.c_double), ("method", ctypes.c_int),
                ("lambda0", ctypes.c_double), ("tail_exact", ctypes.c_int),
                ("tail_window", ctypes.c_double), ("tail_cap_tol", ctypes.c_double)]


class wf_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("stages", ctypes.c_int),
                ("converged", ctypes.c_int), ("refinements", ctypes.c_int),
                ("alpha", ctypes.c_double), ("final_cauchy", ctypes.c_double),
                ("err_estimate", ctypes.c_double), ("fp_residual", ctypes.c_double),
                ("elapsed_ms", ctypes.c_double), ("kernel_launches", ctypes.c_long)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class _Tuning(ctypes.Structure):
    _fields_ = [("syn_np", ctypes.c_int * 2), ("syn_packed", ctypes.c_int),
                ("ana_np", ctypes.c_int * 2), ("ana_queue", ctypes.c_int),
                ("ana_packed", ctypes.c_int), ("ana_global_acc", ctypes.c_int),
                ("syn_ms", (ctypes.c_float * 6) * 2),
                ("ana_ms", (ctypes.c_float * 15) * 2)]


_lib = None
_P = ctypes.c_void_p


def lib():
    """Load libwf.so.  There is no fallback: a missing library is an error."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"libwf.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        I, D = ctypes.c_int, ctypes.c_double
        sigs = {
            "wf_opts_default": (None, [ctypes.POINTER(wf_opts)]),
            "wf_plan": (I, [ctypes.POINTER(_P), I, I, _P, _P, _P,
                            ctypes.POINTER(wf_opts), _P]),
            "wf_set_noise": (I, [_P, _P, _P]),
            "wf_set_cl": (I, [_P, _P]),
            "wf_solve": (I, [_P, _P, _P, _P, _P, _P, ctypes.POINTER(wf_stats)]),
            "wf_solve_host": (I, [_P, _P, _P, _P, ctypes.POINTER(wf_stats)]),
            "wf_residual": (I, [_P, _P, _P, ctypes.POINTER(D), ctypes.POINTER(D),
                                ctypes.POINTER(D)]),
            "wf_solve_batch": (I, [ctypes.POINTER(_P), I, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                   ctypes.POINTER(_P), ctypes.POINTER(wf_stats),
                                   ctypes.POINTER(D)]),
            "wf_residual_static": (I, [_P, _P, _P, ctypes.POINTER(D), ctypes.POINTER(D),
                                       ctypes.POINTER(D)]),
            "wf_alm2map": (I, [_P, _P, _P]),
            "wf_map2alm": (I, [_P, _P, _P]),
            "wf_alm2map_f32": (I, [_P, _P, _P]),
            "wf_map2alm_f32": (I, [_P, _P, _P]),
            "wf_alm2map_df64": (I, [_P, _P, _P]),
            "wf_map2alm_df64": (I, [_P, _P, _P]),
            "wf_map2alm_group": (I, [_P, I, _P, _P]),
            "wf_alm2map_group": (I, [_P, I, _P, _P]),
            "wf_group_stats": (I, [_P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_long),
                                   ctypes.POINTER(D), ctypes.POINTER(D), I]),
            "wf_npix": (ctypes.c_long, [I]),
            "wf_nalm": (ctypes.c_long, [I]),
            "wf_trace": (I, [_P, ctypes.POINTER(I), _P, _P, _P, _P]),
            "wf_kernel_stats": (I, [_P, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_long),
                                    ctypes.POINTER(D), I]),
            "wf_legendre_terms": (I, [_P, I, ctypes.POINTER(D)]),
            "wf_pcg": (I, [_P, _P, _P, _P, D, I, I, I, ctypes.POINTER(wf_stats)]),
            "wf_flat_plan": (I, [ctypes.POINTER(_P), I, D, _P, _P, ctypes.POINTER(wf_opts), _P]),
            "wf_flat_solve": (I, [_P, _P, _P, ctypes.POINTER(wf_stats)]),
            "wf_flat_trace": (I, [_P, ctypes.POINTER(I), _P, _P]),
            "wf_flat_destroy": (None, [_P]),
            "wf_alu_peak": (I, [I, I, ctypes.POINTER(D), ctypes.POINTER(D),
                                ctypes.POINTER(I)]),
            "wf_get_tuning": (I, [_P, ctypes.POINTER(_Tuning)]),
            "wf_set_tuning": (I, [_P, ctypes.POINTER(_Tuning)]),
            "wf_net_create": (I, [ctypes.POINTER(_P), _P, I, I, I, I]),
            "wf_net_num_params": (ctypes.c_long, [_P]),
            "wf_net_set_params": (I, [_P, _P, ctypes.c_long]),
            "wf_net_get_params": (I, [_P, _P, ctypes.c_long]),
            "wf_net_forward": (I, [_P, _P, _P, _P]),
            "wf_net_loss_grad": (I, [_P, _P, _P, ctypes.POINTER(D), _P]),
            "wf_net_adam_step": (I, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float]),
            "wf_net_destroy": (None, [_P]),
            "wf_destroy": (None, [_P]),
            "wf_status_str": (ctypes.c_char_p, [I]),
            "wf_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != WF_OK:
        raise WFError(status, lib().wf_last_error().decode())
    return status


def _dev_ptr(t, dtype, numel, name):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or t.numel() != numel or not t.is_contiguous():
        raise ValueError(f"{name}: expected contiguous {dtype} with {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def wf_opts_default(**overrides):
    o = wf_opts()
    lib().wf_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def wf_npix(nside):
    return 12 * nside * nside


def wf_nalm(lmax):
    return (lmax + 1) * (lmax + 2) // 2


def wf_status_str(s):
    return lib().wf_status_str(int(s)).decode()


def wf_last_error():
    return lib().wf_last_error().decode()


class Plan:
    """A plan: geometry tables, noise, spectrum and workspaces on the GPU."""

    def __init__(self, nside, lmax, cl, noise_var=None, mask=None, opts=None,
                 stream=None, **opt_overrides):
        import torch
        self.nside, self.lmax = int(nside), int(lmax)
        self.npix, self.nalm = wf_npix(nside), wf_nalm(lmax)
        cl = np.ascontiguousarray(cl, dtype=np.float64)
        if cl.shape != (self.lmax + 1,):
            raise ValueError("cl must have lmax + 1 entries")
        self._cl = cl
        if opts is None:
            opts = wf_opts_default(**opt_overrides)
        self.opts = opts
        nv = _dev_ptr(noise_var, torch.float64, self.npix, "noise_var")
        mk = None
        if mask is not None:
            mask = mask.to(torch.uint8).contiguous()
            mk = _dev_ptr(mask, torch.uint8, self.npix, "mask")
        self._stream_obj = stream
        h = ctypes.c_void_p()
        _check(lib().wf_plan(ctypes.byref(h), self.nside, self.lmax,
                             cl.ctypes.data_as(ctypes.c_void_p), nv, mk,
                             ctypes.byref(opts), _stream(stream)))
        self.handle = h

    # -- calls of the C ABI ------------------------------------------------
    def set_noise(self, noise_var, mask=None):
        import torch
        nv = _dev_ptr(noise_var, torch.float64, self.npix, "noise_var")
        mk = None
        if mask is not None:
            mask = mask.to(torch.uint8).contiguous()
            mk = _dev_ptr(mask, torch.uint8, self.npix, "mask")
        _check(lib().wf_set_noise(self.handle, nv, mk))

    def set_cl(self, cl):
        cl = np.ascontiguousarray(cl, dtype=np.float64)
        if cl.shape != (self.lmax + 1,):  # the library reads lmax + 1 values
            raise ValueError("cl must have lmax + 1 entries")
        _check(lib().wf_set_cl(self.handle, cl.ctypes.data_as(ctypes.c_void_p)))
        self._cl = cl

    def solve(self, d, alm=None, map=None, init_alm=None, init_map=None,
              want_map=True, check=True):
        """Returns (alm, map, stats); alm/map are allocated when not given."""
        import torch
        dev = d.device
        if alm is None:
            alm = torch.empty(self.nalm, dtype=torch.complex128, device=dev)
        if map is None and want_map:
            map = torch.empty(self.npix, dtype=torch.float64, device=dev)
        st = wf_stats()
        status = lib().wf_solve(
            self.handle, _dev_ptr(d, torch.float64, self.npix, "d"),
            _dev_ptr(alm, torch.complex128, self.nalm, "alm"),
            _dev_ptr(map, torch.float64, self.npix, "map"),
            _dev_ptr(init_alm, torch.complex128, self.nalm, "init_alm"),
            _dev_ptr(init_map, torch.float64, self.npix, "init_map"),
            ctypes.byref(st))
        if check and status not in (WF_OK,):
            _check(status)
        return alm, map, st.as_dict() | {"status": status}

    def pcg(self, d, tol=1e-6, stop_rule=WF_PCG_STOP_CAUCHY, max_iter=20000, restart=200,
            want_alm=True, want_map=True):
        """wf_pcg: the Wiener filter by preconditioned conjugate gradients
        (App. C).  Returns (alm or None, map or None, stats dict)."""
        import torch
        dev = d.device
        alm = torch.empty(self.nalm, dtype=torch.complex128, device=dev) if want_alm else None
        mp = torch.empty(self.npix, dtype=torch.float64, device=dev) if want_map else None
        st = wf_stats()
        status = lib().wf_pcg(self.handle, _dev_ptr(d, torch.float64, self.npix, "d"),
                              _dev_ptr(alm, torch.complex128, self.nalm, "alm"),
                              _dev_ptr(mp, torch.float64, self.npix, "map"),
                              float(tol), int(stop_rule), int(max_iter), int(restart),
                              ctypes.byref(st))
        if status not in (WF_OK, WF_ERR_NOT_CONVERGED):
            _check(status)
        return alm, mp, st.as_dict() | {"status": status}

    def solve_host(self, d_host, want_alm=True, want_map=True):
        d = np.ascontiguousarray(d_host, dtype=np.float64)
        if d.shape != (self.npix,):  # the library reads Npix values
            raise ValueError("d_host must have Npix entries")
        alm = np.empty(self.nalm, dtype=np.complex128) if want_alm else None
        mp = np.empty(self.npix, dtype=np.float64) if want_map else None
        st = wf_stats()
        status = lib().wf_solve_host(
            self.handle, d.ctypes.data_as(ctypes.c_void_p),
            alm.ctypes.data_as(ctypes.c_void_p) if alm is not None else None,
            mp.ctypes.data_as(ctypes.c_void_p) if mp is not None else None,
            ctypes.byref(st))
        if status != WF_OK:
            _check(status)
        return alm, mp, st.as_dict()

    def residual(self, d, alm):
        import torch
        r1, r2, c2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().wf_residual(self.handle,
                                 _dev_ptr(d, torch.float64, self.npix, "d"),
                                 _dev_ptr(alm, torch.complex128, self.nalm, "alm"),
                                 ctypes.byref(r1), ctypes.byref(r2), ctypes.byref(c2)))
        return {"rel_res_wf": r1.value, "rel_res_fp": r2.value, "chi2": c2.value}

    def residual_static(self, d, alm):
        """wf_residual without allocation during the call (see include/wf.h):
        for callers under a fixed device-memory budget or a pool allocator
        they do not own, and loops that must not stall on cudaMalloc.
        Host-synchronous; must not overlap other calls on this plan.  Small
        plans only."""
        import torch
        r1, r2, c2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().wf_residual_static(
            self.handle, _dev_ptr(d, torch.float64, self.npix, "d"),
            _dev_ptr(alm, torch.complex128, self.nalm, "alm"),
            ctypes.byref(r1), ctypes.byref(r2), ctypes.byref(c2)))
        return {"rel_res_wf": r1.value, "rel_res_fp": r2.value, "chi2": c2.value}

    def alm2map(self, alm, out=None):
        import torch
        if out is None:
            out = torch.empty(self.npix, dtype=torch.float64, device=alm.device)
        _check(lib().wf_alm2map(self.handle,
                                _dev_ptr(alm, torch.complex128, self.nalm, "alm"),
                                _dev_ptr(out, torch.float64, self.npix, "map")))
        return out

    def map2alm(self, m, out=None):
        import torch
        if out is None:
            out = torch.empty(self.nalm, dtype=torch.complex128, device=m.device)
        _check(lib().wf_map2alm(self.handle,
                                _dev_ptr(m, torch.float64, self.npix, "map"),
                                _dev_ptr(out, torch.complex128, self.nalm, "alm")))
        return out

    def alm2map_f32(self, alm, out=None):
        import torch
        if out is None:
            out = torch.empty(self.npix, dtype=torch.float64, device=alm.device)
        _check(lib().wf_alm2map_f32(self.handle,
                                    _dev_ptr(alm, torch.complex128, self.nalm, "alm"),
                                    _dev_ptr(out, torch.float64, self.npix, "map")))
        return out

    def map2alm_f32(self, m, out=None):
        import torch
        if out is None:
            out = torch.empty(self.nalm, dtype=torch.complex128, device=m.device)
        _check(lib().wf_map2alm_f32(self.handle,
                                    _dev_ptr(m, torch.float64, self.npix, "map"),
                                    _dev_ptr(out, torch.complex128, self.nalm, "alm")))
        return out

    def alm2map_df64(self, alm, out=None):
        import torch
        if out is None:
            out = torch.empty(self.npix, dtype=torch.float64, device=alm.device)
        _check(lib().wf_alm2map_df64(self.handle,
                                     _dev_ptr(alm, torch.complex128, self.nalm, "alm"),
                                     _dev_ptr(out, torch.float64, self.npix, "map")))
        return out

    def map2alm_df64(self, m, out=None):
        import torch
        if out is None:
            out = torch.empty(self.nalm, dtype=torch.complex128, device=m.device)
        _check(lib().wf_map2alm_df64(self.handle,
                                     _dev_ptr(m, torch.float64, self.npix, "map"),
                                     _dev_ptr(out, torch.complex128, self.nalm, "alm")))
        return out

    def map2alm_group(self, maps, out=None):
        """alm of each row of maps ([nmaps, npix] float64) in one grouped
        pass (tensor-core Legendre contraction); returns [nmaps, nalm]."""
        import torch
        nm = maps.shape[0]
        if out is None:
            out = torch.empty((nm, self.nalm), dtype=torch.complex128, device=maps.device)
        _check(lib().wf_map2alm_group(self.handle, int(nm),
                                      _dev_ptr(maps, torch.float64, nm * self.npix, "maps"),
                                      _dev_ptr(out, torch.complex128, nm * self.nalm, "alm")))
        return out

    def alm2map_group(self, alm, out=None):
        """maps of each row of alm ([nmaps, nalm] complex128) in one grouped
        pass; returns [nmaps, npix]."""
        import torch
        nm = alm.shape[0]
        if out is None:
            out = torch.empty((nm, self.npix), dtype=torch.float64, device=alm.device)
        _check(lib().wf_alm2map_group(self.handle, int(nm),
                                      _dev_ptr(alm, torch.complex128, nm * self.nalm, "alm"),
                                      _dev_ptr(out, torch.float64, nm * self.npix, "maps")))
        return out

    def group_stats(self, reset=False):
        ms, n = ctypes.c_double(), ctypes.c_long()
        gf, gb = ctypes.c_double(), ctypes.c_double()
        _check(lib().wf_group_stats(self.handle, ctypes.byref(ms), ctypes.byref(n),
                                    ctypes.byref(gf), ctypes.byref(gb), int(reset)))
        return {"ms": ms.value, "launches": n.value, "gflop": gf.value, "gbytes": gb.value}

    def trace(self, cap=1 << 20):
        n = ctypes.c_int(cap)
        st = np.empty(cap, dtype=np.int32)
        xi, mu, c = np.empty(cap), np.empty(cap), np.empty(cap)
        _check(lib().wf_trace(self.handle, ctypes.byref(n),
                              st.ctypes.data_as(ctypes.c_void_p),
                              xi.ctypes.data_as(ctypes.c_void_p),
                              mu.ctypes.data_as(ctypes.c_void_p),
                              c.ctypes.data_as(ctypes.c_void_p)))
        k = n.value
        return {"stage": st[:k], "xi": xi[:k], "mu": mu[:k], "cauchy": c[:k]}

    def kernel_stats(self, kernel=0, reset=False):
        ms, n, gf = ctypes.c_double(), ctypes.c_long(), ctypes.c_double()
        _check(lib().wf_kernel_stats(self.handle, int(kernel), ctypes.byref(ms),
                                     ctypes.byref(n), ctypes.byref(gf), int(reset)))
        key = "gbytes" if int(kernel) in (2, 5) else "gflop"
        return {"ms": ms.value, "launches": n.value, key: gf.value}

    def tuning(self):
        """Launch variants in use and the autotuner's timings (wf_get_tuning)."""
        t = _Tuning()
        _check(lib().wf_get_tuning(self.handle, ctypes.byref(t)))
        return {"syn_np": list(t.syn_np), "syn_packed": t.syn_packed,
                "ana_np": list(t.ana_np), "ana_queue": t.ana_queue,
                "ana_packed": t.ana_packed, "ana_global_acc": t.ana_global_acc,
                "syn_ms": [list(r) for r in t.syn_ms], "ana_ms": [list(r) for r in t.ana_ms]}

    def set_tuning(self, syn_np=None, ana_np=None, ana_queue=None, syn_packed=None,
                   ana_packed=None, ana_global_acc=None):
        """Force launch variants (wf_set_tuning); None keeps the current one."""
        t = _Tuning()
        _check(lib().wf_get_tuning(self.handle, ctypes.byref(t)))
        if syn_np is not None:
            t.syn_np[0], t.syn_np[1] = syn_np
        if ana_np is not None:
            t.ana_np[0], t.ana_np[1] = ana_np
        if ana_queue is not None:
            t.ana_queue = int(ana_queue)
        if syn_packed is not None:
            t.syn_packed = int(syn_packed)
        if ana_packed is not None:
            t.ana_packed = int(ana_packed)
        if ana_global_acc is not None:
            t.ana_global_acc = int(ana_global_acc)
        _check(lib().wf_set_tuning(self.handle, ctypes.byref(t)))

    def legendre_terms(self, L=None):
        t = ctypes.c_double()
        _check(lib().wf_legendre_terms(self.handle, self.lmax if L is None else int(L),
                                       ctypes.byref(t)))
        return t.value

    def close(self):
        if getattr(self, "handle", None):
            lib().wf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def wf_solve_batch(plans, ds, want_alm=True, want_map=False, check=True):
    """Solve several independent problems together (one plan per map).
    Returns (alms, maps, stats list, elapsed_ms)."""
    import torch
    n = len(plans)
    if len(ds) != n:
        raise ValueError("one data map per plan")
    alms = [torch.empty(p.nalm, dtype=torch.complex128, device=d.device) if want_alm else None
            for p, d in zip(plans, ds)]
    maps = [torch.empty(p.npix, dtype=torch.float64, device=d.device) if want_map else None
            for p, d in zip(plans, ds)]
    P = (_P * n)(*[p.handle for p in plans])
    D = (_P * n)(*[_dev_ptr(d, torch.float64, p.npix, "d") for p, d in zip(plans, ds)])
    A = (_P * n)(*[(_dev_ptr(a, torch.complex128, p.nalm, "alm") if a is not None else None)
                   for p, a in zip(plans, alms)])
    M = (_P * n)(*[(_dev_ptr(m, torch.float64, p.npix, "map") if m is not None else None)
                   for p, m in zip(plans, maps)])
    st = (wf_stats * n)()
    ms = ctypes.c_double()
    status = lib().wf_solve_batch(P, n, D, A, M, st, ctypes.byref(ms))
    if check and status != WF_OK:
        _check(status)
    return alms, maps, [s.as_dict() for s in st], ms.value


class Net:
    """The warm-start network of a plan (include/wf.h, wf_net_*)."""

    def __init__(self, plan, channels=16, kernel=9, hidden=32, bf16=True):
        h = ctypes.c_void_p()
        _check(lib().wf_net_create(ctypes.byref(h), plan.handle, int(channels), int(kernel),
                                   int(hidden), int(bool(bf16))))
        self.handle, self.plan = h, plan
        self.channels, self.kernel, self.hidden = channels, kernel, hidden
        self.nparams = int(lib().wf_net_num_params(h))

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib().wf_net_set_params(self.handle, theta.ctypes.data_as(ctypes.c_void_p),
                                       theta.size))

    def get_params(self):
        out = np.empty(self.nparams, dtype=np.float32)
        _check(lib().wf_net_get_params(self.handle, out.ctypes.data_as(ctypes.c_void_p),
                                       out.size))
        return out

    def forward(self, d):
        import torch
        p = self.plan
        t0 = torch.empty(p.npix, dtype=torch.float64, device=d.device)
        a0 = torch.empty(p.nalm, dtype=torch.complex128, device=d.device)
        _check(lib().wf_net_forward(self.handle, _dev_ptr(d, torch.float64, p.npix, "d"),
                                    _dev_ptr(t0, torch.float64, p.npix, "t0"),
                                    _dev_ptr(a0, torch.complex128, p.nalm, "a0")))
        return t0, a0

    def loss_grad(self, d, target, want_grad=False):
        import torch
        p = self.plan
        loss = ctypes.c_double()
        g = np.empty(self.nparams, dtype=np.float32) if want_grad else None
        _check(lib().wf_net_loss_grad(
            self.handle, _dev_ptr(d, torch.float64, p.npix, "d"),
            _dev_ptr(target, torch.complex128, p.nalm, "target"), ctypes.byref(loss),
            g.ctypes.data_as(ctypes.c_void_p) if g is not None else None))
        return loss.value, g

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().wf_net_adam_step(self.handle, float(lr), float(beta1), float(beta2),
                                      float(eps)))

    def close(self):
        if getattr(self, "handle", None):
            lib().wf_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -- functional names of the C ABI ------------------------------------------
def wf_plan(nside, lmax, cl, noise_var=None, mask=None, opts=None, stream=None,
            **opt_overrides):
    return Plan(nside, lmax, cl, noise_var, mask, opts, stream, **opt_overrides)


def wf_solve(plan, d, **kw):
    return plan.solve(d, **kw)


def wf_solve_host(plan, d_host, **kw):
    return plan.solve_host(d_host, **kw)


def wf_residual(plan, d, alm):
    return plan.residual(d, alm)


def wf_alm2map(plan, alm, out=None):
    return plan.alm2map(alm, out)


def wf_map2alm(plan, m, out=None):
    return plan.map2alm(m, out)


def wf_alm2map_f32(plan, alm, out=None):
    return plan.alm2map_f32(alm, out)


def wf_map2alm_f32(plan, m, out=None):
    return plan.map2alm_f32(m, out)


def wf_map2alm_group(plan, maps, out=None):
    return plan.map2alm_group(maps, out)


def wf_alm2map_group(plan, alm, out=None):
    return plan.alm2map_group(alm, out)


def wf_group_stats(plan, reset=False):
    return plan.group_stats(reset)


def wf_alm2map_df64(plan, alm, out=None):
    return plan.alm2map_df64(alm, out)


def wf_map2alm_df64(plan, m, out=None):
    return plan.map2alm_df64(m, out)


def wf_set_noise(plan, noise_var, mask=None):
    return plan.set_noise(noise_var, mask)


def wf_set_cl(plan, cl):
    return plan.set_cl(cl)


def wf_trace(plan):
    return plan.trace()


def wf_kernel_stats(plan, kernel=0, reset=False):
    return plan.kernel_stats(kernel, reset)


class FlatPlan:
    """Algorithm 2 on the flat sky (wf_flat_plan / wf_flat_solve): an n x n
    periodic grid with 2-D FFTs.  ck: host array (n, n) of C at each DFT
    mode (numpy fft2 order); noise_var: CUDA float64 tensor (n, n) or n*n."""

    def __init__(self, n, pixel_area, ck, noise_var, stream=None, **opt_overrides):
        import torch
        self.n = int(n)
        self.opts = wf_opts_default(**opt_overrides)
        ck = np.ascontiguousarray(np.asarray(ck, dtype=np.float64).reshape(-1))
        if ck.size != self.n * self.n:
            raise ValueError("ck: expected n*n values")
        h = _P()
        _check(lib().wf_flat_plan(ctypes.byref(h), self.n, float(pixel_area),
                                  ck.ctypes.data_as(ctypes.c_void_p),
                                  _dev_ptr(noise_var.reshape(-1), torch.float64,
                                           self.n * self.n, "noise_var"),
                                  ctypes.byref(self.opts), _stream(stream)))
        self.handle = h

    def solve(self, d, out=None, check=True):
        import torch
        n2 = self.n * self.n
        if out is None:
            out = torch.empty(n2, dtype=torch.float64, device=d.device)
        st = wf_stats()
        status = lib().wf_flat_solve(self.handle,
                                     _dev_ptr(d.reshape(-1), torch.float64, n2, "d"),
                                     _dev_ptr(out.reshape(-1), torch.float64, n2, "s"),
                                     ctypes.byref(st))
        if check and status != WF_OK:
            _check(status)
        return out.reshape(self.n, self.n), st.as_dict() | {"status": status}

    def trace(self, cap=1 << 20):
        n = ctypes.c_int(cap)
        st, c = np.empty(cap, dtype=np.int32), np.empty(cap)
        _check(lib().wf_flat_trace(self.handle, ctypes.byref(n),
                                   st.ctypes.data_as(ctypes.c_void_p),
                                   c.ctypes.data_as(ctypes.c_void_p)))
        return {"stage": st[:n.value], "cauchy": c[:n.value]}

    def close(self):
        if getattr(self, "handle", None):
            lib().wf_flat_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def wf_alu_peak(kind, reps=5):
    """Measured FMA-pipe peak of the current device: kind 0 = FP64, 1 = FP32,
    2 = packed FP32.  Returns (tflops, best_ms, num_sms)."""
    t, ms, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(lib().wf_alu_peak(int(kind), int(reps), ctypes.byref(t), ctypes.byref(ms),
                             ctypes.byref(n)))
    return t.value, ms.value, n.value


def wf_legendre_terms(plan, L=None):
    return plan.legendre_terms(L)


def wf_get_tuning(plan):
    return plan.tuning()


def wf_set_tuning(plan, syn_np=None, ana_np=None, ana_queue=None, syn_packed=None,
                  ana_packed=None, ana_global_acc=None):
    return plan.set_tuning(syn_np, ana_np, ana_queue, syn_packed, ana_packed, ana_global_acc)


def wf_destroy(plan):
    plan.close()
