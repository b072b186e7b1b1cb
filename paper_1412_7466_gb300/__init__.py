"""Python binding of libgsolve (the C-ABI declared in include/gsolve.h).

Argument marshalling only: every step of the computation runs in the library's CUDA kernels.
Device vectors are torch complex128 tensors on the context's device; host inputs are numpy or
Python sequences.  Importing this package does not load the library; creating a GratingSolver
does, and raises if libgsolve.so has not been built (``python -m paper_1412_7466_gb300.build``)
or no CUDA device is present -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsolve.so")

GS_OK = 0
GS_ERR_ARG = 1
GS_ERR_STATE = 2
GS_ERR_CUDA = 3
GS_ERR_OOM = 4
GS_ERR_GEOMETRY = 5
GS_ERR_NOT_CONVERGED = 6
GS_ERR_NUMERIC = 7
GS_ERR_TIMEOUT = 8
GS_FP64 = 0
GS_C64 = 1
GS_MIXED_BF16 = 3
GS_PROBE_F32X2 = 2
GS_TC_BF16 = 3
GS_TM = 0
GS_TE = 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p


class gs_layers(ctypes.Structure):
    _fields_ = [("d", ctypes.c_double), ("h1_0", ctypes.c_double), ("h2_0", ctypes.c_double),
                ("n_fourier", ctypes.c_int),
                ("h1_cos", _dp), ("h1_sin", _dp), ("h2_cos", _dp), ("h2_sin", _dp),
                ("k1", ctypes.c_double), ("k2", ctypes.c_double), ("k3", ctypes.c_double),
                ("N", ctypes.c_int), ("y0", ctypes.c_double),
                ("Q1", ctypes.c_int), ("Q2", ctypes.c_int), ("Q3", ctypes.c_int),
                ("K_rb", ctypes.c_int),
                ("n_wall1", ctypes.c_int), ("n_wall2", ctypes.c_int), ("n_wall3", ctypes.c_int),
                ("n_bound", ctypes.c_int), ("eps_pinv", ctypes.c_double)]


class gs_inclusions(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("p", ctypes.c_int), ("xy", _dp), ("radius", _dp), ("kp", _dp)]


class gs_star_inclusions(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("p", ctypes.c_int), ("xy", _dp), ("phi", _dp), ("a1", ctypes.c_double),
                ("a2", ctypes.c_double), ("a3", ctypes.c_int), ("kp", ctypes.c_double), ("n_nodes", ctypes.c_int)]


class gs_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("restart", ctypes.c_int),
                ("precision", ctypes.c_int), ("inner_tol", ctypes.c_double), ("max_sweeps", ctypes.c_int)]


_SIGS = {
    "gs_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp]),
    "gs_destroy": (None, [_vp]),
    "gs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "gs_last_error": (ctypes.c_char_p, [_vp]),
    "gs_set_layers": (ctypes.c_int, [_vp, ctypes.POINTER(gs_layers)]),
    "gs_set_incidence": (ctypes.c_int, [_vp, ctypes.c_int, _dp]),
    "gs_set_inclusions": (ctypes.c_int, [_vp, ctypes.POINTER(gs_inclusions)]),
    "gs_set_polarization": (ctypes.c_int, [_vp, ctypes.c_int]),
    "gs_set_inclusions_star": (ctypes.c_int, [_vp, ctypes.POINTER(gs_star_inclusions)]),
    "gs_get_scattering_blocks": (ctypes.c_int, [_vp, _vp]),
    "gs_set_inclusion_loss": (ctypes.c_int, [_vp, _dp]),
    "gs_factor": (ctypes.c_int, [_vp]),
    "gs_dims": (ctypes.c_int, [_vp, _ip, _ip, _ip, _ip, _ip]),
    "gs_get_A": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "gs_get_f": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "gs_get_coupling": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "gs_get_scattering": (ctypes.c_int, [_vp, _vp]),
    "gs_pinv_apply": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "gs_translate": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int]),
    "gs_apply": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int]),
    "gs_rhs": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "gs_solve": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(gs_solve_opts), _vp]),
    "gs_solve_angles": (ctypes.c_int, [_vp, ctypes.POINTER(gs_solve_opts)]),
    "gs_get_beta": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "gs_stats": (ctypes.c_int, [_vp, ctypes.c_int, _ip, _dp]),
    "gs_bragg": (ctypes.c_int, [_vp, ctypes.c_int, _ip, _ip, _vp, _ip, _ip, _vp, _dp]),
    "gs_launch_count": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_ulonglong)]),
    "gs_profile": (ctypes.c_int, [_vp, ctypes.c_int]),
    "gs_profile_read": (ctypes.c_int, [_vp, ctypes.c_int, _ip, _dp]),
    "gs_stats_refinement": (ctypes.c_int, [_vp, ctypes.c_int, _ip]),
    "gs_factor_stats": (ctypes.c_int, [_vp, ctypes.c_int, _ip, _ip, _dp, _vp, _vp, _ip, _dp]),
    "gs_probe_fma": (ctypes.c_int, [_vp, ctypes.c_int, _dp]),
    "gs_set_table_budget": (ctypes.c_int, [_vp, ctypes.c_double]),
    "gs_set_inclusions_batch": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(gs_inclusions)]),
    "gs_factor_batch": (ctypes.c_int, [_vp]),
    "gs_apply_batch": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int]),
    "gs_solve_batch": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(gs_solve_opts)]),
    "gs_batch_stats": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _ip, _dp]),
    "gs_get_beta_batch": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp]),
    "gs_bragg_batch": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _ip, _ip, _vp, _ip, _ip, _vp, _dp]),
    "gs_batch_tuning": (ctypes.c_int, [_vp, _ip, _ip]),
    "gs_translate_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, _vp, _vp, ctypes.c_int, _vp]),
    "gs_tc_gemm_bf16": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_long, ctypes.c_long, ctypes.c_long]),
    "gs_translate_multi": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "gs_translate_multi_split": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "gs_field": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_long, _vp, _vp]),
    "gs_mlp_param_count": (ctypes.c_int, [ctypes.c_int]),
    "gs_mlp_set_params": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_long]),
    "gs_mlp_get_params": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_long]),
    "gs_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_long, _vp]),
    "gs_mlp_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_long, _vp, _dp]),
    "gs_mlp_train_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_long, ctypes.c_double, _dp]),
    "gs_ws_features": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "gs_ws_targets": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "gs_ws_moments": (ctypes.c_int, [_vp, ctypes.c_int, _dp]),
    "gs_ws_normalise": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double]),
    "gs_warm_start": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _dp, _ip]),
}

_lib = None


def exported_symbols():
    """Names of the C-ABI functions this binding expects the library to export."""
    return sorted(_SIGS)


def load_library(path: str = LIB_PATH):
    """Loads libgsolve.so (raises if it has not been built) and declares the signatures."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_1412_7466_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def translate_noalloc(xy, beta, out, p, k2, d, alpha, precision=GS_FP64, stream=None):
    """alpha = T beta through the allocation-free entry point (no context; for callers that
    cannot allocate device memory).  xy: (M, 2) float64, beta and out: M (2p+1) complex128, all
    contiguous CUDA tensors on the current device, out not overlapping beta or xy (the library
    trusts these sizes, so they are checked here).  Returns the status code."""
    import torch
    lib = load_library()
    if not (isinstance(xy, torch.Tensor) and xy.dtype == torch.float64 and xy.dim() == 2 and xy.shape[1] == 2):
        raise ValueError("xy must be a (M, 2) float64 tensor")
    n = int(xy.shape[0]) * (2 * int(p) + 1)
    for name, t in (("beta", beta), ("out", out)):
        if not (isinstance(t, torch.Tensor) and t.dtype == torch.complex128 and t.numel() == n):
            raise ValueError(f"{name} must be a complex128 tensor of M (2p+1) = {n} values")
    dev = torch.cuda.current_device()
    for name, t in (("xy", xy), ("beta", beta), ("out", out)):
        if not t.is_cuda or t.device.index != dev or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous tensor on the current CUDA device ({dev})")

    def span(t):
        a = t.data_ptr()
        return a, a + t.numel() * t.element_size()

    o0, o1 = span(out)
    for t in (beta, xy):
        a0, a1 = span(t)
        if t.numel() and out.numel() and a0 < o1 and o0 < a1:
            raise ValueError("out overlaps an input")
    st = stream if stream is not None else torch.cuda.current_stream()
    a = complex(alpha)
    return lib.gs_translate_noalloc(int(xy.shape[0]), int(p), _vp(xy.data_ptr()), float(k2), float(d), a.real,
                                    a.imag, _vp(beta.data_ptr()), _vp(out.data_ptr()), int(precision),
                                    _vp(st.cuda_stream))


class GsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _arr(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a, a.ctypes.data_as(_dp)


class GratingSolver:
    """One gsolve context on a CUDA device (torch's current stream at creation)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("GratingSolver needs a CUDA device (there is no CPU fallback)")
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = _vp()
        self._check(self.lib.gs_create(ctypes.byref(h), device, _vp(stream.cuda_stream)), "gs_create", ctx=None)
        self.ctx = h
        self._keep = []

    # -- plumbing ------------------------------------------------------------------------------
    def _check(self, st, what, ctx="self", ok=(GS_OK,)):
        if st in ok:
            return st
        c = self.ctx if ctx == "self" else None
        detail = self.lib.gs_last_error(c).decode() if c else ""
        raise GsError(st, f"{what}: {self.lib.gs_strerror(st).decode()} {detail}")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.gs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _cvec(self, n):
        return self.torch.empty(n, dtype=self.torch.complex128, device=self.device)

    def _as_dev(self, x):
        t = self.torch.as_tensor(x)
        return t.to(device=self.device, dtype=self.torch.complex128).contiguous()

    # -- problem definition ---------------------------------------------------------------------
    def set_layers(self, g: dict):
        nf = max(len(g["gamma1"].get("cos", [])), len(g["gamma1"].get("sin", [])),
                 len(g["gamma2"].get("cos", [])), len(g["gamma2"].get("sin", [])))

        def pad(v):
            v = list(v) + [0.0] * (nf - len(v))
            return _arr(v if nf else [0.0])

        arrs = [pad(g["gamma1"].get("cos", [])), pad(g["gamma1"].get("sin", [])),
                pad(g["gamma2"].get("cos", [])), pad(g["gamma2"].get("sin", []))]
        self._keep = [a for a, _ in arrs]
        L = gs_layers(d=g["d"], h1_0=g["gamma1"]["h0"], h2_0=g["gamma2"]["h0"], n_fourier=nf,
                      h1_cos=arrs[0][1], h1_sin=arrs[1][1], h2_cos=arrs[2][1], h2_sin=arrs[3][1],
                      k1=g["k"][0], k2=g["k"][1], k3=g["k"][2], N=g["N"], y0=g["y0"],
                      Q1=g["Q"][0], Q2=g["Q"][1], Q3=g["Q"][2], K_rb=g["K_rb"],
                      n_wall1=g["n_wall"][0], n_wall2=g["n_wall"][1], n_wall3=g["n_wall"][2],
                      n_bound=g["n_bound"], eps_pinv=g["eps_pinv"])
        self._check(self.lib.gs_set_layers(self.ctx, ctypes.byref(L)), "gs_set_layers")
        pol = g.get("pol", "TM")
        if pol not in ("TM", "TE"):
            raise ValueError("polarisation must be 'TM' or 'TE'")
        self._check(self.lib.gs_set_polarization(self.ctx, GS_TE if pol == "TE" else GS_TM), "gs_set_polarization")
        self.grating = g

    def set_incidence(self, thetas):
        a, p = _arr(np.atleast_1d(thetas))
        self._check(self.lib.gs_set_incidence(self.ctx, a.size, p), "gs_set_incidence")
        self.thetas = a.copy()

    def set_inclusions(self, disks: dict):
        """Disks {"xy", "radius", "kp", "p"}; a complex kp (Im kp >= 0) makes the disks lossy.  With
        "shape": {"a1", "a2", "a3", "N"} and "phi" (rotation per inclusion), rotated stars of that
        shape and interior wavenumber kp[0] (gs_set_inclusions_star)."""
        if "shape" in disks:
            sh = disks["shape"]
            xy, pxy = _arr(disks["xy"])
            ph, pph = _arr(disks["phi"])
            I = gs_star_inclusions(M=xy.shape[0], p=int(disks["p"]), xy=pxy, phi=pph, a1=float(sh["a1"]),
                                   a2=float(sh["a2"]), a3=int(sh["a3"]), kp=float(np.real(disks["kp"][0])),
                                   n_nodes=int(sh["N"]))
            self._check(self.lib.gs_set_inclusions_star(self.ctx, ctypes.byref(I)), "gs_set_inclusions_star")
            self.M, self.p = xy.shape[0], int(disks["p"])
            return
        xy, pxy = _arr(disks["xy"])
        r, pr = _arr(disks["radius"])
        kpc = np.asarray(disks["kp"])
        kp, pkp = _arr(np.real(kpc))
        I = gs_inclusions(M=xy.shape[0], p=int(disks["p"]), xy=pxy, radius=pr, kp=pkp)
        self._check(self.lib.gs_set_inclusions(self.ctx, ctypes.byref(I)), "gs_set_inclusions")
        if np.iscomplexobj(kpc) and np.any(np.imag(kpc) != 0):
            ki, pki = _arr(np.imag(kpc))
            self._check(self.lib.gs_set_inclusion_loss(self.ctx, pki), "gs_set_inclusion_loss")
        self.M, self.p = xy.shape[0], int(disks["p"])

    def factor(self):
        self._check(self.lib.gs_factor(self.ctx), "gs_factor")

    def dims(self):
        v = [ctypes.c_int() for _ in range(5)]
        self._check(self.lib.gs_dims(self.ctx, *[ctypes.byref(x) for x in v]), "gs_dims")
        return dict(zip(("rows", "cols", "n", "nB", "nC"), [x.value for x in v]))

    # -- inspection -----------------------------------------------------------------------------
    def get_A(self, angle=0):
        d = self.dims()
        t = self._cvec(d["rows"] * d["cols"])
        self._check(self.lib.gs_get_A(self.ctx, angle, _ptr(t)), "gs_get_A")
        return t.view(d["cols"], d["rows"]).T     # column-major storage

    def get_f(self, angle=0):
        t = self._cvec(self.dims()["rows"])
        self._check(self.lib.gs_get_f(self.ctx, angle, _ptr(t)), "gs_get_f")
        return t

    def get_coupling(self, angle=0):
        d = self.dims()
        B = self._cvec(d["n"] * d["nB"])
        Cm = self._cvec(d["nC"] * d["n"])
        self._check(self.lib.gs_get_coupling(self.ctx, angle, _ptr(B), _ptr(Cm)), "gs_get_coupling")
        return B.view(d["n"], d["nB"]), Cm.view(d["nC"], d["n"])

    def get_scattering_blocks(self):
        """(M, 2p+1, 2p+1) blocks of the preconditioner (the rotated star matrices, or diagonal)."""
        nc = 2 * self.p + 1
        t = self._cvec(self.M * nc * nc)
        self._check(self.lib.gs_get_scattering_blocks(self.ctx, _ptr(t)), "gs_get_scattering_blocks")
        return t.view(self.M, nc, nc)

    def get_scattering(self):
        t = self._cvec(self.dims()["n"])
        self._check(self.lib.gs_get_scattering(self.ctx, _ptr(t)), "gs_get_scattering")
        return t.view(self.M, 2 * self.p + 1)

    def pinv_apply(self, g, angle=0):
        g = self._as_dev(g)
        x = self._cvec(self.dims()["cols"])
        self._check(self.lib.gs_pinv_apply(self.ctx, angle, _ptr(g), _ptr(x)), "gs_pinv_apply")
        return x

    # -- hot path -------------------------------------------------------------------------------
    def translate(self, beta, angle=0, precision=GS_FP64, out=None):
        beta = self._as_dev(beta)
        out = self._cvec(beta.numel()) if out is None else out
        self._check(self.lib.gs_translate(self.ctx, angle, _ptr(beta), _ptr(out), precision), "gs_translate")
        return out

    def apply(self, x, angle=0, precision=GS_FP64, out=None):
        x = self._as_dev(x)
        out = self._cvec(x.numel()) if out is None else out
        self._check(self.lib.gs_apply(self.ctx, angle, _ptr(x), _ptr(out), precision), "gs_apply")
        return out

    def rhs(self, angle=0):
        b = self._cvec(self.dims()["n"])
        self._check(self.lib.gs_rhs(self.ctx, angle, _ptr(b)), "gs_rhs")
        return b

    def solve(self, angle=0, tol=1e-11, maxit=4000, restart=500, precision=GS_FP64, beta0=None,
              allow_unconverged=False, inner_tol=1e-6, max_sweeps=0):
        o = gs_solve_opts(tol=tol, maxit=maxit, restart=restart, precision=precision, inner_tol=inner_tol,
                          max_sweeps=max_sweeps)
        b0 = _ptr(self._as_dev(beta0)) if beta0 is not None else None
        ok = (GS_OK, GS_ERR_NOT_CONVERGED) if allow_unconverged else (GS_OK,)
        return self._check(self.lib.gs_solve(self.ctx, angle, ctypes.byref(o), b0), "gs_solve", ok=ok)

    def solve_angles(self, tol=1e-11, maxit=4000, restart=500, inner_tol=1e-6, max_sweeps=0,
                     allow_unconverged=False, precision=None):
        """All incidence angles of the context in lockstep (mixed form); precision GS_C64 (default:
        each angle from the complex64 pair table) or GS_MIXED_BF16 (the translation of all angles at
        once on the tensor cores); per-angle results through stats/get_beta/bragg(angle)."""
        o = gs_solve_opts(tol=tol, maxit=maxit, restart=restart,
                          precision=GS_C64 if precision is None else precision, inner_tol=inner_tol,
                          max_sweeps=max_sweeps)
        ok = (GS_OK, GS_ERR_NOT_CONVERGED) if allow_unconverged else (GS_OK,)
        return self._check(self.lib.gs_solve_angles(self.ctx, ctypes.byref(o)), "gs_solve_angles", ok=ok)

    def refinement_sweeps(self, angle=0):
        v = ctypes.c_int()
        self._check(self.lib.gs_stats_refinement(self.ctx, angle, ctypes.byref(v)), "gs_stats_refinement")
        return v.value

    def factor_stats(self, angle=0):
        """Sweeps and per-phase device times (ms) of the angle's grating factorisation."""
        s32, s64, ph = ctypes.c_int(), ctypes.c_int(), (ctypes.c_double * 6)()
        r32, r64 = (ctypes.c_longlong * 32)(), (ctypes.c_longlong * 32)()
        nss, nsd = ctypes.c_int(), (ctypes.c_double * 6)()
        self._check(self.lib.gs_factor_stats(self.ctx, angle, ctypes.byref(s32), ctypes.byref(s64), ph, r32, r64,
                                             ctypes.byref(nss), nsd), "gs_factor_stats")
        names = ("assemble", "qr", "jacobi_fp32", "polar_step", "jacobi_fp64", "u_v")
        return {"sweeps_fp32": s32.value, "sweeps_fp64": s64.value, "phase_ms": dict(zip(names, list(ph))),
                "rotations_fp32": list(r32)[:s32.value], "rotations_fp64": list(r64)[:s64.value],
                "newton_schulz_steps": nss.value, "newton_schulz_defects": list(nsd)[:min(nss.value + 1, 6)]}

    def get_beta(self, angle=0):
        t = self._cvec(self.dims()["n"])
        self._check(self.lib.gs_get_beta(self.ctx, angle, _ptr(t)), "gs_get_beta")
        return t

    def stats(self, angle=0):
        it, rr = ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.gs_stats(self.ctx, angle, ctypes.byref(it), ctypes.byref(rr)), "gs_stats")
        return it.value, rr.value

    def set_table_budget(self, gb):
        self._check(self.lib.gs_set_table_budget(self.ctx, float(gb)), "gs_set_table_budget")

    # -- batched solves (many geometries on one grating) -----------------------------------------
    def set_inclusions_batch(self, geos):
        keep, arr = [], (gs_inclusions * len(geos))()
        for q, dk in enumerate(geos):
            xy, pxy = _arr(dk["xy"])
            r, pr = _arr(dk["radius"])
            kp, pkp = _arr(dk["kp"])
            keep += [xy, r, kp]
            arr[q] = gs_inclusions(M=xy.shape[0], p=int(dk["p"]), xy=pxy, radius=pr, kp=pkp)
        self._check(self.lib.gs_set_inclusions_batch(self.ctx, len(geos), arr), "gs_set_inclusions_batch")
        self.batch_sizes = [np.asarray(dk["xy"]).shape[0] * (2 * int(dk["p"]) + 1) for dk in geos]
        self.p = int(geos[0]["p"])

    def factor_batch(self):
        self._check(self.lib.gs_factor_batch(self.ctx), "gs_factor_batch")

    def apply_batch(self, x, angle=0, precision=GS_FP64):
        x = self._as_dev(x)
        y = self._cvec(x.numel())
        self._check(self.lib.gs_apply_batch(self.ctx, angle, _ptr(x), _ptr(y), precision), "gs_apply_batch")
        return y

    def solve_batch(self, angle=0, tol=1e-11, maxit=4000, restart=500, precision=GS_FP64, inner_tol=1e-6,
                    max_sweeps=0, allow_unconverged=False):
        o = gs_solve_opts(tol=tol, maxit=maxit, restart=restart, precision=precision, inner_tol=inner_tol,
                          max_sweeps=max_sweeps)
        ok = (GS_OK, GS_ERR_NOT_CONVERGED) if allow_unconverged else (GS_OK,)
        return self._check(self.lib.gs_solve_batch(self.ctx, angle, ctypes.byref(o)), "gs_solve_batch", ok=ok)

    def batch_stats(self, g, angle=0):
        it, rr = ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.gs_batch_stats(self.ctx, angle, g, ctypes.byref(it), ctypes.byref(rr)), "gs_batch_stats")
        return it.value, rr.value

    def get_beta_batch(self, g, angle=0):
        t = self._cvec(self.batch_sizes[g])
        self._check(self.lib.gs_get_beta_batch(self.ctx, angle, g, _ptr(t)), "gs_get_beta_batch")
        return t

    def bragg_batch(self, g, angle=0):
        cap = 2 * self.grating["K_rb"] + 1
        nt, nb = ctypes.c_int(), ctypes.c_int()
        ot = (ctypes.c_int * cap)()
        ob = (ctypes.c_int * cap)()
        c = np.zeros(cap, dtype=np.complex128)
        d = np.zeros(cap, dtype=np.complex128)
        fe = ctypes.c_double()
        self._check(self.lib.gs_bragg_batch(self.ctx, angle, g, ctypes.byref(nt), ot, c.ctypes.data_as(_vp),
                                            ctypes.byref(nb), ob, d.ctypes.data_as(_vp), ctypes.byref(fe)),
                    "gs_bragg_batch")
        return {"n_top": np.array(ot[:nt.value]), "c": c[:nt.value].copy(),
                "n_bot": np.array(ob[:nb.value]), "d": d[:nb.value].copy(), "flux_err": fe.value}

    def batch_tuning(self):
        ch, bp = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.gs_batch_tuning(self.ctx, ctypes.byref(ch), ctypes.byref(bp)), "gs_batch_tuning")
        return ch.value, bp.value

    # -- instrumentation ------------------------------------------------------------------------
    def launch_count(self):
        v = ctypes.c_ulonglong()
        self._check(self.lib.gs_launch_count(self.ctx, ctypes.byref(v)), "gs_launch_count")
        return v.value

    def profile(self, enable=True):
        self._check(self.lib.gs_profile(self.ctx, int(bool(enable))), "gs_profile")

    def profile_read(self, precision=GS_FP64):
        n, ms = ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.gs_profile_read(self.ctx, precision, ctypes.byref(n), ctypes.byref(ms)),
                    "gs_profile_read")
        return n.value, ms.value

    # -- learned warm start ---------------------------------------------------------------------
    def _fdev(self, x, cols):
        t = self.torch.as_tensor(x).to(device=self.device, dtype=self.torch.float32).contiguous()
        if t.dim() != 2 or t.shape[1] != cols:
            raise ValueError(f"expected a (rows, {cols}) array")
        return t

    def mlp_param_count(self, p):
        n = self.lib.gs_mlp_param_count(int(p))
        if n < 0:
            raise ValueError("unsupported multipole order")
        return n

    def mlp_set_params(self, p, params):
        a = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        self._check(self.lib.gs_mlp_set_params(self.ctx, int(p), a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               a.size), "gs_mlp_set_params")
        self._mlp_p = int(p)

    def mlp_get_params(self):
        a = np.empty(self.mlp_param_count(self._mlp_p), dtype=np.float32)
        self._check(self.lib.gs_mlp_get_params(self.ctx, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size),
                    "gs_mlp_get_params")
        return a

    def mlp_forward(self, X):
        X = self._fdev(X, 64)
        Y = self.torch.empty(X.shape[0], 2 * (2 * self._mlp_p + 1), dtype=self.torch.float32, device=self.device)
        self._check(self.lib.gs_mlp_forward(self.ctx, _ptr(X), X.shape[0], _ptr(Y)), "gs_mlp_forward")
        return Y

    def mlp_loss_grad(self, X, Y):
        X, Y = self._fdev(X, 64), self._fdev(Y, 2 * (2 * self._mlp_p + 1))
        nw = self.mlp_param_count(self._mlp_p) - 128 - (2 * self._mlp_p + 1)
        g = self.torch.empty(nw, dtype=self.torch.float32, device=self.device)
        loss = ctypes.c_double()
        self._check(self.lib.gs_mlp_loss_grad(self.ctx, _ptr(X), _ptr(Y), X.shape[0], _ptr(g), ctypes.byref(loss)),
                    "gs_mlp_loss_grad")
        return loss.value, g

    def mlp_train_step(self, X, Y, lr):
        """One Adam step; X, Y must already be float32 device tensors of shapes (rows, 64), (rows, 2(2p+1))."""
        loss = ctypes.c_double()
        self._check(self.lib.gs_mlp_train_step(self.ctx, _ptr(X), _ptr(Y), X.shape[0], float(lr), ctypes.byref(loss)),
                    "gs_mlp_train_step")
        return loss.value

    def ws_features(self, angle=0):
        X = self.torch.empty(self.dims()["n"] // (2 * self._mlp_p + 1), 64, dtype=self.torch.float32,
                             device=self.device)
        self._check(self.lib.gs_ws_features(self.ctx, angle, _ptr(X)), "gs_ws_features")
        return X

    def ws_targets(self, angle=0):
        nc = 2 * self._mlp_p + 1
        Y = self.torch.empty(self.dims()["n"] // nc, 2 * nc, dtype=self.torch.float32, device=self.device)
        self._check(self.lib.gs_ws_targets(self.ctx, angle, _ptr(Y)), "gs_ws_targets")
        return Y

    def ws_moments(self, angle=0):
        """(mean |t_n|^2, mean |s_n t_n|^2) per order from the last solution."""
        ms = np.empty(2 * (2 * self._mlp_p + 1))
        self._check(self.lib.gs_ws_moments(self.ctx, angle, ms.ctypes.data_as(_dp)), "gs_ws_moments")
        nc = 2 * self._mlp_p + 1
        return ms[:nc], ms[nc:]

    def ws_normalise(self, theta_range, k_range, share=1e-4, angle=0):
        """Fixes the network's feature standardisation and per-order output scale from the current
        geometry and its last solution at `angle` (gs_ws_normalise)."""
        self._check(self.lib.gs_ws_normalise(self.ctx, angle, float(theta_range[0]), float(theta_range[1]),
                                             float(k_range[0]), float(k_range[1]), float(share)), "gs_ws_normalise")

    def warm_start(self, angle=0):
        """(beta_0 device tensor, its relative residual, used); beta_0 is zero when not used."""
        b0 = self._cvec(self.dims()["n"])
        rel, used = ctypes.c_double(), ctypes.c_int()
        self._check(self.lib.gs_warm_start(self.ctx, angle, _ptr(b0), ctypes.byref(rel), ctypes.byref(used)),
                    "gs_warm_start")
        return b0, rel.value, bool(used.value)

    def field(self, pts, angle=0):
        """Total field in the middle layer at points pts ((npts, 2) array) from the last solution;
        NaN outside one period of the layer or inside an inclusion.  Returns a complex128 tensor."""
        P = self.torch.as_tensor(pts).to(device=self.device, dtype=self.torch.float64).contiguous()
        if P.dim() != 2 or P.shape[1] != 2:
            raise ValueError("pts must be (npts, 2)")
        u = self._cvec(P.shape[0])
        self._check(self.lib.gs_field(self.ctx, angle, P.shape[0], _ptr(P), _ptr(u)), "gs_field")
        return u

    def translate_multi(self, alphas, betas):
        """Translations of R right-hand sides (rows of betas, (R, n) complex) with image phases
        alphas (R complex), on the tensor cores (bfloat16 in, FP32 accumulate); returns (R, n)."""
        a = np.ascontiguousarray(np.asarray(alphas, dtype=np.complex128))
        B = self._as_dev(betas)
        if B.dim() != 2 or B.shape[0] != a.size:
            raise ValueError("betas must be (R, n) with R = len(alphas)")
        out = self.torch.empty_like(B)
        self._check(self.lib.gs_translate_multi(self.ctx, a.size, a.ctypes.data_as(_vp), _ptr(B), _ptr(out)),
                    "gs_translate_multi")
        return out

    def translate_multi_split(self, alphas, betas):
        """As translate_multi with the operator and the coefficients each split into three bfloat16
        parts (single-precision accuracy): the inner operator of solve_angles."""
        a = np.ascontiguousarray(np.asarray(alphas, dtype=np.complex128))
        B = self._as_dev(betas)
        if B.dim() != 2 or B.shape[0] != a.size:
            raise ValueError("betas must be (R, n) with R = len(alphas)")
        out = self.torch.empty_like(B)
        self._check(self.lib.gs_translate_multi_split(self.ctx, a.size, a.ctypes.data_as(_vp), _ptr(B), _ptr(out)),
                    "gs_translate_multi_split")
        return out

    def tc_gemm_bf16(self, A, B):
        """C = A B^T on the tensor cores: A (M, K) and B (N, K) bfloat16 device tensors, C (M, N) FP32."""
        A = A.contiguous()
        B = B.contiguous()
        C = self.torch.empty(A.shape[0], B.shape[0], dtype=self.torch.float32, device=self.device)
        self._check(self.lib.gs_tc_gemm_bf16(self.ctx, _ptr(A), _ptr(B), _ptr(C), A.shape[0], B.shape[0], A.shape[1]),
                    "gs_tc_gemm_bf16")
        return C

    def probe_fma(self, precision=GS_FP64):
        v = ctypes.c_double()
        self._check(self.lib.gs_probe_fma(self.ctx, precision, ctypes.byref(v)), "gs_probe_fma")
        return v.value

    def bragg(self, angle=0):
        cap = 2 * self.grating["K_rb"] + 1
        nt, nb = ctypes.c_int(), ctypes.c_int()
        ot = (ctypes.c_int * cap)()
        ob = (ctypes.c_int * cap)()
        c = np.zeros(cap, dtype=np.complex128)
        d = np.zeros(cap, dtype=np.complex128)
        fe = ctypes.c_double()
        self._check(self.lib.gs_bragg(self.ctx, angle, ctypes.byref(nt), ot, c.ctypes.data_as(_vp),
                                      ctypes.byref(nb), ob, d.ctypes.data_as(_vp), ctypes.byref(fe)),
                    "gs_bragg")
        return {"n_top": np.array(ot[:nt.value]), "c": c[:nt.value].copy(),
                "n_bot": np.array(ob[:nb.value]), "d": d[:nb.value].copy(), "flux_err": fe.value}
