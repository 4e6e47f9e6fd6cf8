"""ctypes binding of libpprpa_gb300.so (argument marshalling only).

Every entry point of include/pprpa.h has a same-named function here.  Array
arguments are either NumPy float64 arrays (host) or torch CUDA float64
tensors (device); the binding checks dtype/contiguity, passes raw pointers
and converts a negative return code into :class:`PprpaError`.  No step of
the computation runs in Python.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpprpa_gb300.so")

OK = 0
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NOCONV, ERR_UNSTABLE, ERR_TIMEOUT, ERR_STATE, ERR_UNSUPPORTED = (
    -1, -2, -3, -4, -5, -6, -7, -8)
HOST, DEVICE = 0, 1
SINGLET, TRIPLET = 1, 3
AB = 2  # alpha-beta subspace of spin-unrestricted ppRPA (after Context.set_beta)
METHOD_FULL, METHOD_DAVIDSON = 0, 1
PREC_FP64, PREC_BF16, PREC_FP8 = 0, 1, 2
PREC_BF16_SPLIT = PREC_BF16 + 16  # sigma only: BF16x3 split products
CHANNEL_PP, CHANNEL_HH = 0, 1  # lowest N+2 roots / highest N-2 roots


class Options(ctypes.Structure):
    _fields_ = [
        ("mult", ctypes.c_int),
        ("channel", ctypes.c_int),
        ("method", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("nroots", ctypes.c_int),
        ("conv_tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("max_subspace", ctypes.c_int),
        ("want_ec", ctypes.c_int),
        ("require_definite", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("iters_stage1", ctypes.c_int),
        ("n_sigma", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("max_resid", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("max_imag", ctypes.c_double),
        ("t_sigma_ms", ctypes.c_double),
        ("t_total_ms", ctypes.c_double),
        ("sigma_flops", ctypes.c_double),
        ("nconv", ctypes.c_int),
        ("n_real", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PprpaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# name -> (restype, argtypes); mirrors include/pprpa.h
SIGNATURES = {
    "pprpa_create": (_I, [ctypes.POINTER(_P), _I, _P]),
    "pprpa_destroy": (None, [_P]),
    "pprpa_set_orbitals": (_I, [_P, _I, _P, _P]),
    "pprpa_set_active": (_I, [_P, _I, _I]),
    "pprpa_set_ao": (_I, [_P, _I, _I, _P, _P, _I]),
    "pprpa_set_mo": (_I, [_P, _I, _P, _I]),
    "pprpa_get_L": (_I, [_P, _P, _I]),
    "pprpa_dims": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                        ctypes.POINTER(_I)]),
    "pprpa_diag": (_I, [_P, _I, _P, _I]),
    "pprpa_sigma": (_I, [_P, _I, _I, _I, _P, _P, _I]),
    "pprpa_build_matrix": (_I, [_P, _I, _P, _I]),
    "pprpa_solve": (_I, [_P, ctypes.POINTER(Options), _P, _P, _P, _P, ctypes.POINTER(Info)]),
    "pprpa_grad": (_I, [_P, _I, _P, _P, _I]),
    "pprpa_grad_vector": (_I, [_P, _I, _P, _P, _P, _I]),
    "pprpa_grad_ec": (_I, [_P, _P, _P, _I]),
    "pprpa_grad_sum": (_I, [_P, _I, _P, _P, _P, _I]),
    "pprpa_grad_ao": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _I]),
    "pprpa_analyze": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _I]),
    "pprpa_set_beta": (_I, [_P, _I, _I, _I, _P, _P, _I]),
    "pprpa_grad_ab": (_I, [_P, _I, _P, _P, _P, _P, _I]),
    "pprpa_strerror": (ctypes.c_char_p, [_I]),
    "pprpa_last_error": (ctypes.c_char_p, []),
    "pprpa_kernel_launches": (ctypes.c_longlong, []),
    "pprpa_profile": (_I, [_P, _I, _P]),
    "pprpa_sigma_noalloc": (_I, [_I, _I, _I, _I, _P, _P, _I, _P, _P, _P]),
    "pprpa_sigma_batch": (_I, [_I, _P, _P, _P, _P, _P, _I, _I]),
    "pprpa_autotune": (_I, [_P, _I, _I, _I, _P]),
    "pprpa_solve_batch": (_I, [_I, _P, _P, _P, _P, _P, _P, _P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != OK:
        lib = load()
        raise PprpaError(rc, f"{lib.pprpa_strerror(rc).decode()}: {lib.pprpa_last_error().decode()}")
    return rc


def _ptr(a, writable=False):
    """(pointer, where) of a float64 NumPy array or torch tensor."""
    if a is None:
        return None, HOST
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("host arrays must be C-contiguous float64")
        if writable and not a.flags["WRITEABLE"]:
            raise TypeError("output array is read-only")
        return a.ctypes.data, HOST
    # torch tensor
    import torch

    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr(), (DEVICE if a.is_cuda else HOST)
    raise TypeError(f"unsupported array type {type(a)}")


def _need(a, shape, what):
    """The library reads and writes exactly these extents through raw pointers: refuse any
    other shape before the call."""
    if a is not None and tuple(a.shape) != tuple(shape):
        raise ValueError(f"{what}: expected shape {tuple(shape)}, got {tuple(a.shape)}")


def _vectors(z, N, what):
    """k of a (k, N) block or of one (N,) vector."""
    if z.ndim == 1:
        _need(z, (N,), what)
        return 1
    if z.ndim != 2 or z.shape[1] != N:
        raise ValueError(f"{what}: expected shape (k, {N}) or ({N},), got {tuple(z.shape)}")
    return int(z.shape[0])


def pair_counts(nocc_act, nvir_act, mult):
    """(nvv, noo) of the restricted pair lists: a <= b for singlets, a < b for triplets."""
    if mult == SINGLET:
        return nvir_act * (nvir_act + 1) // 2, nocc_act * (nocc_act + 1) // 2
    if mult == TRIPLET:
        return nvir_act * (nvir_act - 1) // 2, nocc_act * (nocc_act - 1) // 2
    raise ValueError("mult must be SINGLET or TRIPLET")


def sigma_batch(contexts, mults, zs, outs, precision=PREC_BF16, graph=True):
    """Batched sigma over molecules (pprpa_sigma_batch); zs / outs are CUDA tensors."""
    n = len(contexts)
    if not (len(mults) == len(zs) == len(outs) == n):
        raise ValueError("sigma_batch: one mult, z and out per context")
    for c, m, z, o in zip(contexts, mults, zs, outs):
        _, _, nvv, noo = c.dims(m)
        _vectors(z, nvv + noo, "sigma_batch z")
        _need(o, z.shape, "sigma_batch out")
    ctxs = (_P * n)(*[c._h.value for c in contexts])
    mu = (_I * n)(*[int(m) for m in mults])
    ks = (_I * n)(*[int(z.shape[0]) for z in zs])
    zp = (_P * n)(*[z.data_ptr() for z in zs])
    op = (_P * n)(*[o.data_ptr() for o in outs])
    _check(load().pprpa_sigma_batch(n, ctxs, mu, ks, zp, op, int(precision), 1 if graph else 0))
    return outs


def solve_batch(contexts, mults, nroots, precision=PREC_BF16, conv_tol=1e-5, max_iter=200,
                channel=CHANNEL_PP, max_subspace=0, require_definite=False):
    """pprpa_solve_batch over several contexts (one molecule each, one device).

    mults / nroots: one entry per molecule (or a single value for all).  Returns a list of
    dicts like Context.solve (omega, X, Y, info, rc); raises only for a call-level argument
    error, a molecule's own failure shows in its rc."""
    n = len(contexts)
    mults = list(mults) if hasattr(mults, "__len__") else [mults] * n
    nroots = list(nroots) if hasattr(nroots, "__len__") else [nroots] * n
    opts = (Options * n)()
    om, Xs, Ys = [], [], []
    for m, c in enumerate(contexts):
        _, _, nvv, noo = c.dims(mults[m])
        opts[m] = Options(int(mults[m]), int(channel), METHOD_DAVIDSON, int(precision), int(nroots[m]),
                          float(conv_tol), int(max_iter), int(max_subspace), 0, int(require_definite))
        om.append(np.empty(nroots[m]))
        Xs.append(np.empty((nroots[m], nvv)))
        Ys.append(np.empty((nroots[m], max(noo, 1))))
    infos = (Info * n)()
    rcs = (_I * n)()
    ctxs = (_P * n)(*[c._h for c in contexts])
    po = (_P * n)(*[a.ctypes.data for a in om])
    px = (_P * n)(*[a.ctypes.data for a in Xs])
    py = (_P * n)(*[a.ctypes.data for a in Ys])
    rc = load().pprpa_solve_batch(n, ctxs, opts, po, px, py, infos, rcs)
    if rc == ERR_ARG and all(r == 0 for r in rcs):
        _check(rc)
    out = []
    for m, c in enumerate(contexts):
        if rcs[m] in (OK, ERR_NOCONV):
            c._last_mult = mults[m]
        noo = c.dims(mults[m])[3]
        out.append({"omega": om[m], "X": Xs[m], "Y": Ys[m][:, :noo], "info": infos[m].as_dict(),
                    "rc": int(rcs[m])})
    return out


def sigma_noalloc(mult, nocc_act, nvir_act, L, eps, z, out, stream=None):
    """FP64 sigma without any device allocation (pprpa_sigma_noalloc).

    For callers that cannot allocate device memory; all arrays are CUDA float64
    tensors on the current device and the work is only enqueued on ``stream``.
    """
    import torch

    dev = torch.cuda.current_device()
    for a in (L, eps, z, out):
        p, w = _ptr(a)
        if w != DEVICE:
            raise TypeError("sigma_noalloc takes device tensors only")
        if a.device.index != dev:
            # the library runs on the current device and looks up its scratch there
            raise ValueError(f"sigma_noalloc: tensor on cuda:{a.device.index}, current device is cuda:{dev}")
    n = int(nocc_act) + int(nvir_act)
    _need(L, (L.shape[0], n, n), "sigma_noalloc L")
    _need(eps, (n,), "sigma_noalloc eps")
    k = _vectors(z, sum(pair_counts(int(nocc_act), int(nvir_act), int(mult))), "sigma_noalloc z")
    _need(out, z.shape, "sigma_noalloc out")
    _check(load().pprpa_sigma_noalloc(int(mult), int(nocc_act), int(nvir_act), int(L.shape[0]),
                                      L.data_ptr(), eps.data_ptr(), k, z.data_ptr(),
                                      out.data_ptr(), stream))
    return out


def kernel_launches() -> int:
    return int(load().pprpa_kernel_launches())


class Context:
    """Owns one pprpa_ctx (library-owned device memory, one CUDA stream)."""

    def __init__(self, device: int = 0, stream=None):
        lib = load()
        h = _P()
        _check(lib.pprpa_create(ctypes.byref(h), int(device), stream))
        self._h = h
        self.lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self.lib.pprpa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- inputs ----
    def set_orbitals(self, occ, eps):
        occ = np.ascontiguousarray(occ, dtype=np.float64)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        if occ.shape != eps.shape or occ.ndim != 1:
            raise ValueError("occ and eps must be 1-D of equal length")
        _check(self.lib.pprpa_set_orbitals(self._h, occ.shape[0], occ.ctypes.data, eps.ctypes.data))
        self._nmo = int(occ.shape[0])

    def set_active(self, nocc_act, nvir_act):
        _check(self.lib.pprpa_set_active(self._h, int(nocc_act), int(nvir_act)))

    def set_ao(self, C, ao3c):
        pc, wc = _ptr(C)
        pa, wa = _ptr(ao3c)
        if wc != wa:
            raise ValueError("C and ao3c must both be host or both be device arrays")
        naux, nb, nb2 = ao3c.shape
        if nb != nb2 or C.shape[0] != nb:
            raise ValueError("shape mismatch between C and ao3c")
        _need(C, (nb, getattr(self, "_nmo", C.shape[1])), "set_ao C (nbasis x nmo of set_orbitals)")
        _check(self.lib.pprpa_set_ao(self._h, nb, naux, pc, pa, wa))

    def set_beta(self, nocc_b, nvir_b, eps_b, L_b):
        """Beta active space of a spin-unrestricted reference (the context's own is alpha):
        energies eps_b[nb] and MO-space integrals L_b[naux][nb][nb], occupied first."""
        pe, we = _ptr(eps_b)
        pl, wl = _ptr(L_b)
        if we != wl:
            raise ValueError("eps_b and L_b must both be host or both be device arrays")
        nb = int(nocc_b) + int(nvir_b)
        _need(eps_b, (nb,), "set_beta eps_b")
        _need(L_b, (L_b.shape[0], nb, nb), "set_beta L_b")
        _check(self.lib.pprpa_set_beta(self._h, int(nocc_b), int(nvir_b), int(L_b.shape[0]), pe, pl, wl))
        self._nb = int(nocc_b) + int(nvir_b)
        self._nob, self._nvb = int(nocc_b), int(nvir_b)

    def set_mo(self, L):
        nmo = getattr(self, "_nmo", L.shape[1])
        _need(L, (L.shape[0], nmo, nmo), "set_mo L (naux x nmo x nmo of set_orbitals)")
        p, w = _ptr(L)
        _check(self.lib.pprpa_set_mo(self._h, L.shape[0], p, w))

    def dims(self, mult):
        n, naux, nvv, noo = _I(), _I(), _I(), _I()
        _check(self.lib.pprpa_dims(self._h, int(mult), ctypes.byref(n), ctypes.byref(naux),
                                   ctypes.byref(nvv), ctypes.byref(noo)))
        return n.value, naux.value, nvv.value, noo.value

    def get_L(self, out=None):
        n, naux, _, _ = self.dims(1)
        if out is None:
            out = np.empty((naux, n, n))
        _need(out, (naux, n, n), "get_L out")
        p, w = _ptr(out, True)
        _check(self.lib.pprpa_get_L(self._h, p, w))
        return out

    # ---- kernels ----
    def diag(self, mult, out=None):
        _, _, nvv, noo = self.dims(mult)
        if out is None:
            out = np.empty(nvv + noo)
        _need(out, (nvv + noo,), "diag out")
        p, w = _ptr(out, True)
        _check(self.lib.pprpa_diag(self._h, int(mult), p, w))
        return out

    def sigma(self, mult, z, precision=PREC_FP64, out=None):
        pz, wz = _ptr(z)
        _, _, nvv, noo = self.dims(mult)
        k = _vectors(z, nvv + noo, "sigma z")
        if out is None:
            out = np.empty_like(z) if isinstance(z, np.ndarray) else z.new_empty(z.shape)
        _need(out, z.shape, "sigma out")
        po, wo = _ptr(out, True)
        if wz != wo:
            raise ValueError("z and out must live on the same side")
        _check(self.lib.pprpa_sigma(self._h, int(mult), int(precision), int(k), pz, po, wz))
        return out

    def build_matrix(self, mult, out=None):
        _, _, nvv, noo = self.dims(mult)
        N = nvv + noo
        if out is None:
            out = np.empty((N, N))
        _need(out, (N, N), "build_matrix out")
        p, w = _ptr(out, True)
        _check(self.lib.pprpa_build_matrix(self._h, int(mult), p, w))
        return out

    # ---- solve / gradient ----
    def solve(self, mult=SINGLET, nroots=10, method=METHOD_DAVIDSON, precision=PREC_FP64,
              conv_tol=1e-6, max_iter=200, max_subspace=0, want_ec=False, raise_noconv=True,
              channel=CHANNEL_PP, require_definite=False):
        """pp channel: the lowest N+2 roots, ascending, X^T X - Y^T Y = +1.
        hh channel: the highest N-2 roots, descending, X^T X - Y^T Y = -1."""
        _, _, nvv, noo = self.dims(mult)
        o = Options(mult, channel, method, precision, nroots, conv_tol, max_iter, max_subspace,
                    int(want_ec), int(require_definite))
        omega = np.empty(nroots)
        X = np.empty((nroots, nvv))
        Y = np.empty((nroots, max(noo, 1)))
        ec = np.full(1, np.nan)
        info = Info()
        rc = self.lib.pprpa_solve(self._h, ctypes.byref(o), omega.ctypes.data, X.ctypes.data,
                                  Y.ctypes.data, ec.ctypes.data if want_ec else None,
                                  ctypes.byref(info))
        # a Davidson solve that stopped without converging (max_iter, or lowest roots
        # interleaved with complex pairs: UNSTABLE after some iterations with n_real Ritz
        # values) returns its last iterate; one that stopped at its first indefinite subspace
        # (require_definite) returns none.  raise_noconv=False hands either back instead of
        # raising; "iterate" says whether omega / X / Y hold a last iterate.
        davidson = method == METHOD_DAVIDSON
        stopped = rc == ERR_NOCONV or (rc == ERR_UNSTABLE and davidson and info.iters > 0
                                       and info.n_real > 0)
        if rc == OK or stopped:
            self._last_mult = mult  # the library now holds this solve's vectors
        if rc != OK and not (davidson and rc in (ERR_NOCONV, ERR_UNSTABLE) and not raise_noconv):
            _check(rc)
        return {"omega": omega, "X": X, "Y": Y[:, :noo], "ec": float(ec[0]),
                "info": info.as_dict(), "rc": rc, "iterate": rc == OK or stopped}

    def autotune(self, mult, k, precision=PREC_BF16):
        """Tune the tensor-core tile widths on this problem; returns the four widths."""
        t = (_I * 4)()
        _check(self.lib.pprpa_autotune(self._h, int(mult), int(k), int(precision), t))
        return list(t)

    def grad_sum(self, w, dL=None, deps=None):
        """Gradient of sum_r w[r] omega_r over the first len(w) roots of the last solve."""
        n, naux, _, _ = self.dims(1)
        wh = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1))
        if dL is None:
            dL = np.empty((naux, n, n))
        if deps is None:
            deps = np.empty(n) if isinstance(dL, np.ndarray) else dL.new_empty(n)
        _need(dL, (naux, n, n), "grad_sum dL")
        _need(deps, (n,), "grad_sum deps")
        p1, w1 = _ptr(dL, True)
        p2, w2 = _ptr(deps, True)
        if w1 != w2:
            raise ValueError("dL and deps must live on the same side")
        _check(self.lib.pprpa_grad_sum(self._h, int(wh.shape[0]), wh.ctypes.data, p1, p2, w1))
        return dL, deps

    def grad_ec(self, dL=None, deps=None):
        """dE_c/dL^P_pq and dE_c/d eps_p after a solve that returned every root of its
        channel (every addition root, or every removal root)."""
        n, naux, _, _ = self.dims(1)
        if dL is None:
            dL = np.empty((naux, n, n))
        if deps is None:
            deps = np.empty(n) if isinstance(dL, np.ndarray) else dL.new_empty(n)
        _need(dL, (naux, n, n), "grad_ec dL")
        _need(deps, (n,), "grad_ec deps")
        p1, w1 = _ptr(dL, True)
        p2, w2 = _ptr(deps, True)
        if w1 != w2:
            raise ValueError("dL and deps must live on the same side")
        _check(self.lib.pprpa_grad_ec(self._h, p1, p2, w1))
        return dL, deps

    def analyze(self, root, ab=None):
        """Two-electron density matrix and NTOs of root `root` of the last solve (host arrays):
        dict with D2e (n x n), lam_p, Cp1, Cp2 (virtual block) and lam_h, Ch1, Ch2 (occupied).
        For a root of the alpha-beta subspace (the last solve had mult = AB; `ab`, if given,
        must agree) D2e is diag(D^alpha, D^beta) and Cp2 / Ch2 run over beta orbitals."""
        last_ab = getattr(self, "_last_mult", None) == AB
        if ab is not None and bool(ab) != last_ab:
            raise ValueError("analyze: `ab` does not match the subspace of the last solve")
        ab = last_ab
        n, _, nvv1, _ = self.dims(1)
        nv = int(round((np.sqrt(8.0 * nvv1 + 1.0) - 1.0) / 2.0))  # singlet nvv = nv (nv + 1) / 2
        no = n - nv
        nob, nvb, nd = no, nv, n
        if ab:
            nob, nvb = getattr(self, "_nob", 0), getattr(self, "_nvb", 0)
            nd = n + nob + nvb
        out = {"D2e": np.empty((nd, nd)), "lam_p": np.empty(nv), "lam_h": np.empty(no),
               "Cp1": np.empty((nv, nv)), "Cp2": np.empty((nvb, nv)),
               "Ch1": np.empty((no, no)), "Ch2": np.empty((nob, no))}
        ptr = lambda a: a.ctypes.data if a.size else None
        _check(self.lib.pprpa_analyze(self._h, int(root), ptr(out["D2e"]), ptr(out["lam_p"]),
                                      ptr(out["lam_h"]), ptr(out["Cp1"]), ptr(out["Cp2"]),
                                      ptr(out["Ch1"]), ptr(out["Ch2"]), HOST))
        return out

    def grad_ao(self, C, dL, ao3c=None, want_dao=True, want_dc=True):
        """Adjoint of the AO->MO transform: (d/d(P|mu nu), d/dC) from d/dL^P_pq.

        Arrays are all host (NumPy) or all device (torch); ``ao3c`` is needed for dC only."""
        n_ = self.dims(1)[0]  # valid before any integrals are set: naux comes from dL
        _need(dL, (dL.shape[0], n_, n_), "grad_ao dL")
        naux, n, _ = dL.shape
        nb, nmo = C.shape
        _need(C, (nb, getattr(self, "_nmo", nmo)), "grad_ao C (nbasis x nmo of set_orbitals)")
        if ao3c is not None:
            _need(ao3c, (naux, nb, nb), "grad_ao ao3c")
        if want_dc and ao3c is None:
            raise ValueError("dC needs ao3c")
        host = isinstance(dL, np.ndarray)
        new = (lambda shape: np.empty(shape)) if host else (lambda shape: dL.new_empty(shape))
        d_ao = new((naux, nb, nb)) if want_dao else None
        d_c = new((nb, nmo)) if want_dc else None
        pc, wc = _ptr(C)
        pl, wl = _ptr(dL)
        pa, wa = _ptr(ao3c) if ao3c is not None else (None, wl)
        po, wo = _ptr(d_ao, True) if d_ao is not None else (None, wl)
        pq, wq = _ptr(d_c, True) if d_c is not None else (None, wl)
        if len({wc, wl, wa, wo, wq}) != 1:
            raise ValueError("every array must live on the same side")
        _check(self.lib.pprpa_grad_ao(self._h, nb, naux, pc, pa, pl, po, pq, wl))
        return d_ao, d_c

    def grad_vector(self, mult, z, dL=None, deps=None):
        """d(z^T M z)/dL^P_pq and d(z^T M z)/d eps_p for an explicit pair vector z."""
        n, naux, _, _ = self.dims(mult)
        if dL is None:
            dL = np.empty((naux, n, n)) if isinstance(z, np.ndarray) else z.new_empty((naux, n, n))
        if deps is None:
            deps = np.empty(n) if isinstance(dL, np.ndarray) else dL.new_empty(n)
        _, _, nvv, noo = self.dims(mult)
        _need(z, (nvv + noo,), "grad_vector z")
        _need(dL, (naux, n, n), "grad_vector dL")
        _need(deps, (n,), "grad_vector deps")
        pz, wz = _ptr(z)
        p1, w1 = _ptr(dL, True)
        p2, w2 = _ptr(deps, True)
        if not (wz == w1 == w2):
            raise ValueError("z, dL and deps must live on the same side")
        _check(self.lib.pprpa_grad_vector(self._h, int(mult), pz, p1, p2, w1))
        return dL, deps

    def profile(self, enable=None):
        """Read the tensor-core GEMM timing records (4 x {launches, ms, flops});
        enable=True/False clears and starts/stops recording after the read."""
        out = np.zeros(12)
        _check(self.lib.pprpa_profile(self._h, -1 if enable is None else int(bool(enable)),
                                      out.ctypes.data))
        return out.reshape(4, 3)

    def grad_ab(self, root):
        """Gradient of alpha-beta root `root` of the last solve (mult = AB): host arrays
        (dLa [naux][na][na], dLb [naux][nb][nb], deps_a [na], deps_b [nb])."""
        na, naux, _, _ = self.dims(1)
        nb = getattr(self, "_nb", 0)
        if nb == 0:
            raise PprpaError(-7, "grad_ab: call set_beta first")
        dLa = np.empty((naux, na, na))
        dLb = np.empty((naux, nb, nb))
        dea = np.empty(na)
        deb = np.empty(nb)
        _check(self.lib.pprpa_grad_ab(self._h, int(root), _ptr(dLa, True)[0], _ptr(dLb, True)[0],
                                      _ptr(dea, True)[0], _ptr(deb, True)[0], HOST))
        return dLa, dLb, dea, deb

    def grad(self, root, dL=None, deps=None):
        n, naux, _, _ = self.dims(1)
        if dL is None:
            dL = np.empty((naux, n, n))
        if deps is None:
            deps = np.empty(n) if isinstance(dL, np.ndarray) else dL.new_empty(n)
        _need(dL, (naux, n, n), "grad dL")
        _need(deps, (n,), "grad deps")
        p1, w1 = _ptr(dL, True)
        p2, w2 = _ptr(deps, True)
        if w1 != w2:
            raise ValueError("dL and deps must live on the same side")
        _check(self.lib.pprpa_grad(self._h, int(root), p1, p2, w1))
        return dL, deps
