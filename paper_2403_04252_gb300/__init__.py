"""GB300 (sm_103a) implementation of the WP-CCC hot path behind a C ABI.

This package is a thin ctypes binding over ``libwpccc.so`` (declared in
``include/wpccc.h``): it marshals numpy inputs and torch CUDA tensors into the
C calls and does no arithmetic of the method itself.  Every step (matrix
elements, solve, RK4 propagation, probabilities) runs in the library's CUDA
kernels; there is no CPU fallback.  If the library has not been built, importing
this package raises.

Matrices are stored column-major (LAPACK layout): a batch of N x N matrices is a
complex128 tensor of shape (batch, N, N) whose memory holds matrix k, column j,
row i at [k, j, i].  ``natural(t)`` returns the (batch, row, column) view.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwpccc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = C.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ESINGULAR, ENONFINITE, ECUDA, EUNSUPPORTED, ETIMEOUT, ENOCONV = range(9)
_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ESINGULAR", 4: "ENONFINITE", 5: "ECUDA", 6: "EUNSUPPORTED",
          7: "ETIMEOUT", 8: "ENOCONV"}
DEFAULT_WAIT_POLLS = 1 << 20
LMAX = 10
NMAX = 8192

_pd = C.POINTER(C.c_double)
_pi = C.POINTER(C.c_int)


class _CentreDesc(C.Structure):
    _fields_ = [("Z", C.c_double), ("n_rad", C.c_int), ("rad_l", _pi), ("f", _pd),
                ("n_states", C.c_int), ("st_rad", _pi), ("st_m", _pi), ("st_eps", _pd)]


class _BasisDesc(C.Structure):
    _fields_ = [("n_centres", C.c_int), ("Nr", C.c_int), ("r", _pd), ("w", _pd),
                ("T", _CentreDesc), ("P", _CentreDesc),
                ("Geta", C.c_int), ("s", _pd), ("ws", _pd),
                ("Gtau", C.c_int), ("tau", _pd), ("wtau", _pd), ("gamma", C.c_double),
                ("mp_c", C.c_double), ("mp_a", C.c_double), ("mp_b", C.c_double)]


class _PathsDesc(C.Structure):
    _fields_ = [("n_paths", C.c_int), ("b", _pd), ("v", _pd), ("n_z", _pi), ("z", _pd)]


_lib.wpccc_basis_create.argtypes = [C.POINTER(_BasisDesc), C.c_int, C.POINTER(C.c_void_p)]
_lib.wpccc_basis_destroy.argtypes = [C.c_void_p]
_lib.wpccc_basis_info.argtypes = [C.c_void_p, _pi, _pi]
_lib.wpccc_matrix_elements.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int, _pd,
                                       C.c_void_p, C.c_void_p, C.c_void_p]
_lib.wpccc_matrix_elements_noalloc.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int, _pd,
                                               C.c_void_p, C.c_void_p, C.c_void_p]
_lib.wpccc_solve.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_int, C.c_void_p]
_lib.wpccc_propagate.argtypes = [C.c_void_p, C.POINTER(_PathsDesc), C.c_int, C.c_int, C.c_void_p, C.c_void_p]
_lib.wpccc_probabilities.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.wpccc_basis_set_workspace_limit.argtypes = [C.c_void_p, C.c_size_t]
_lib.wpccc_profile_enable.argtypes = [C.c_void_p, C.c_int]
_lib.wpccc_basis_set_solve_mode.argtypes = [C.c_void_p, C.c_int]
_lib.wpccc_basis_set_refine_iters.argtypes = [C.c_void_p, C.c_int]
_lib.wpccc_basis_set_rk4_layout.argtypes = [C.c_void_p, C.c_int]
_lib.wpccc_profile_read.argtypes = [C.c_void_p, _pd, C.POINTER(C.c_longlong)]
_lib.wpccc_batch_create.argtypes = [C.c_int, C.POINTER(C.c_void_p), C.POINTER(_PathsDesc), C.c_int,
                                    C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p)]
_lib.wpccc_batch_launch.argtypes = [C.c_void_p, C.c_void_p]
_lib.wpccc_batch_status.argtypes = [C.c_void_p, C.c_void_p]
_lib.wpccc_batch_info.argtypes = [C.c_void_p, _pi, _pd]
_lib.wpccc_batch_destroy.argtypes = [C.c_void_p]
_lib.wpccc_matrix_elements_precision.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int, _pd,
                                                 C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
_lib.wpccc_basis_set_tangents.argtypes = [C.c_void_p, C.c_int, _pd, _pd, _pd, _pd, _pd]
_lib.wpccc_propagate_adjoint.argtypes = [C.c_void_p, C.POINTER(_PathsDesc), C.c_int, _pd, C.c_int, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]
_lib.wpccc_observables.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.wpccc_cross_sections.argtypes = [C.c_int, _pd, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.wpccc_overlap_norms.argtypes = [C.c_void_p, C.c_int, _pd, _pd, _pd, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.wpccc_basis_states.argtypes = [C.c_void_p, _pi, _pd]
_lib.wpccc_basis_set_refine_tolerance.argtypes = [C.c_void_p, C.c_double]
_lib.wpccc_basis_set_wait_limit.argtypes = [C.c_void_p, C.c_long]
_lib.wpccc_basis_set_schur_update.argtypes = [C.c_void_p, C.c_int]
_lib.wpccc_last_error.restype = C.c_char_p
for _f in ("wpccc_basis_create", "wpccc_basis_destroy", "wpccc_basis_info", "wpccc_matrix_elements",
           "wpccc_solve", "wpccc_propagate", "wpccc_probabilities", "wpccc_basis_set_workspace_limit",
           "wpccc_profile_enable", "wpccc_profile_read", "wpccc_basis_set_solve_mode",
           "wpccc_matrix_elements_noalloc", "wpccc_batch_create", "wpccc_batch_launch", "wpccc_batch_status",
           "wpccc_batch_info", "wpccc_batch_destroy", "wpccc_basis_set_tangents", "wpccc_propagate_adjoint",
           "wpccc_matrix_elements_precision", "wpccc_basis_set_refine_iters", "wpccc_basis_set_rk4_layout",
           "wpccc_observables", "wpccc_cross_sections", "wpccc_overlap_norms", "wpccc_basis_states",
           "wpccc_basis_set_refine_tolerance", "wpccc_basis_set_wait_limit", "wpccc_basis_set_schur_update"):
    getattr(_lib, _f).restype = C.c_int

EXPORTED = ("wpccc_basis_create", "wpccc_basis_destroy", "wpccc_basis_info", "wpccc_matrix_elements",
            "wpccc_solve", "wpccc_propagate", "wpccc_probabilities", "wpccc_basis_set_workspace_limit",
            "wpccc_profile_enable", "wpccc_profile_read", "wpccc_basis_set_solve_mode", "wpccc_last_error",
            "wpccc_matrix_elements_noalloc", "wpccc_batch_create", "wpccc_batch_launch", "wpccc_batch_status",
            "wpccc_batch_info", "wpccc_batch_destroy", "wpccc_basis_set_tangents", "wpccc_propagate_adjoint",
            "wpccc_matrix_elements_precision", "wpccc_basis_set_refine_iters", "wpccc_basis_set_rk4_layout",
            "wpccc_observables", "wpccc_cross_sections", "wpccc_overlap_norms", "wpccc_basis_states",
            "wpccc_basis_set_refine_tolerance", "wpccc_basis_set_wait_limit", "wpccc_basis_set_schur_update")
MAX_PARAMS = 4
SCHUR_UPDATE_AUTO, SCHUR_UPDATE_TENSOR, SCHUR_UPDATE_CUDA_CORES = 0, 1, 2
RK4_AUTO, RK4_SHARED, RK4_GLOBAL = 0, 1, 2
MAX_REFINE = 8
NOALLOC_SCRATCH_BYTES = 64 << 20
SOLVE_STAGE, SOLVE_MATRIX, SOLVE_SCHUR = 0, 1, 2
PROF_CATEGORIES = ("node_tables", "mol_gemm", "rotate_direct", "solve", "rk4", "adjoint")


class WpcccError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.wpccc_last_error().decode()
        super().__init__(f"{where}: {_NAMES.get(status, status)}: {msg}")


def _check(status: int, where: str) -> None:
    if status != OK:
        raise WpcccError(status, where)


def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(_pi if dtype == np.int32 else _pd)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _check_matrices(S, H, nz: int, N: int, device: int, where: str) -> None:
    """Refuses, before any launch, output tensors the kernels would write past or misread: both must be
    complex128, contiguous, on the basis' CUDA device and hold at least nz * N * N elements."""
    for name, t in (("S", S), ("H", H)):
        if t is None:
            raise ValueError(f"{where}: {name} is required")
        if str(t.dtype) != "torch.complex128":
            raise ValueError(f"{where}: {name} must be complex128, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{where}: {name} must be contiguous")
        if t.numel() < nz * N * N:
            raise ValueError(f"{where}: {name} holds {t.numel()} elements, {nz} positions of N = {N} need "
                             f"{nz * N * N}")
        if t.device.type != "cuda" or t.device.index != device:
            raise ValueError(f"{where}: {name} is on {t.device}, the basis is on cuda:{device}")


def _check_amplitudes(c, n_paths: int, N: int, device: int, where: str) -> None:
    """Refuses an amplitude tensor the kernels would misread: complex128, contiguous, on the basis' device,
    at least n_paths * N elements."""
    if str(c.dtype) != "torch.complex128":
        raise ValueError(f"{where}: c must be complex128, got {c.dtype}")
    if not c.is_contiguous():
        raise ValueError(f"{where}: c must be contiguous")
    if c.numel() < n_paths * N:
        raise ValueError(f"{where}: c holds {c.numel()} elements, {n_paths} paths of N = {N} need {n_paths * N}")
    if c.device.type != "cuda" or c.device.index != device:
        raise ValueError(f"{where}: c is on {c.device}, the basis is on cuda:{device}")


def natural(t):
    """(batch, row, column) view of column-major matrix storage."""
    return t.transpose(-1, -2)


def colmajor(t):
    """Column-major storage tensor of a (batch, row, column) tensor (a copy)."""
    return t.transpose(-1, -2).contiguous()


class Basis:
    """A basis resident on one CUDA device (``wpccc_basis_create``)."""

    def __init__(self, basis, device: int = 0):
        """`basis` is a ``wpccc_inputs.Basis`` (grid, centres, quadrature, charges)."""
        keep = []

        def arr(a, dt):
            a, p = _arr(a, dt)
            keep.append(a)
            return p

        def centre(c, Z):
            if c is None:
                return _CentreDesc(Z=Z)
            return _CentreDesc(Z=Z, n_rad=int(c.n_rad), rad_l=arr(c.rad_l, np.int32), f=arr(c.f, np.float64),
                               n_states=int(c.N), st_rad=arr(c.st_rad, np.int32), st_m=arr(c.st_m, np.int32),
                               st_eps=arr(c.st_eps, np.float64))

        g = basis.grid
        d = _BasisDesc(n_centres=basis.n_centres, Nr=int(g.r.size), r=arr(g.r, np.float64), w=arr(g.w, np.float64),
                       T=centre(basis.T, basis.Z_T), P=centre(basis.P, basis.Z_P))
        if basis.n_centres == 2:
            q = basis.quad
            d.Geta, d.s, d.ws = int(q.s.size), arr(q.s, np.float64), arr(q.ws, np.float64)
            d.Gtau, d.tau, d.wtau = int(q.tau.size), arr(q.tau, np.float64), arr(q.wtau, np.float64)
            d.gamma = float(q.gamma)
            d.mp_c = float(getattr(basis, "mp_c", 0.0))
            d.mp_a = float(getattr(basis, "mp_a", 0.0))
            d.mp_b = float(getattr(basis, "mp_b", 0.0))
        h = C.c_void_p()
        _check(_lib.wpccc_basis_create(C.byref(d), int(device), C.byref(h)), "wpccc_basis_create")
        self._h = h
        self.device = int(device)
        nt, np_ = C.c_int(), C.c_int()
        _check(_lib.wpccc_basis_info(h, C.byref(nt), C.byref(np_)), "wpccc_basis_info")
        self.N_T, self.N_P = nt.value, np_.value
        self.N = self.N_T + self.N_P
        self.n_centres = basis.n_centres
        self.n_par = 0
        if getattr(basis, "tangent_T", None) is not None:
            self.set_tangents(basis.tangent_T.df, basis.tangent_T.deps, basis.tangent_P.df, basis.tangent_P.deps,
                              basis.dexplicit)

    def set_tangents(self, dfT, depsT, dfP, depsP, dexplicit) -> None:
        """Derivatives of the radial tables and energies of both centres and of (Z_P, mp_c, mp_a, mp_b)
        with respect to each parameter (``wpccc_basis_set_tangents``)."""
        dexplicit = np.atleast_2d(np.asarray(dexplicit, dtype=np.float64))
        n_par = int(dexplicit.shape[0])
        arrs = [_arr(x, np.float64) for x in (dfT, depsT, dfP, depsP, dexplicit)]
        _check(_lib.wpccc_basis_set_tangents(self._h, n_par, *[p for _, p in arrs]), "wpccc_basis_set_tangents")
        self.n_par = n_par

    def close(self):
        if getattr(self, "_h", None):
            _lib.wpccc_basis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_workspace_limit(self, nbytes: int) -> None:
        _check(_lib.wpccc_basis_set_workspace_limit(self._h, C.c_size_t(int(nbytes))),
               "wpccc_basis_set_workspace_limit")

    def set_solve_mode(self, mode: int) -> None:
        """SOLVE_STAGE (LU of S once per position, solve per RK4 stage), SOLVE_SCHUR (Cholesky of the Schur
        complement I - K^+ K once per position, solve per stage) or SOLVE_MATRIX (X = S^-1 H)."""
        _check(_lib.wpccc_basis_set_solve_mode(self._h, int(mode)), "wpccc_basis_set_solve_mode")

    def set_rk4_layout(self, layout: int) -> None:
        """RK4_AUTO (default), RK4_SHARED (one block per path, vectors in shared memory) or RK4_GLOBAL
        (one-centre form: a launch per RK4 stage, vectors in global memory, any N)."""
        _check(_lib.wpccc_basis_set_rk4_layout(self._h, int(layout)), "wpccc_basis_set_rk4_layout")

    def set_refine_iters(self, iters: int) -> None:
        """FP64 refinement sweeps per RK4 stage of the refined precision modes (1, 2, 3, 5); default 2."""
        _check(_lib.wpccc_basis_set_refine_iters(self._h, int(iters)), "wpccc_basis_set_refine_iters")

    def set_refine_tolerance(self, tol: float) -> None:
        """Largest last refinement correction relative to the solution before wpccc_propagate reports
        ENOCONV (refined precision modes; default 1e-3, <= 0 switches the check off)."""
        _check(_lib.wpccc_basis_set_refine_tolerance(self._h, float(tol)), "wpccc_basis_set_refine_tolerance")

    def set_schur_update(self, mode: int) -> None:
        """SCHUR_UPDATE_AUTO (default), _TENSOR or _CUDA_CORES: where the refined Schur forms' FP32
        preconditioner forms I - K^+ K (``wpccc_basis_set_schur_update``)."""
        _check(_lib.wpccc_basis_set_schur_update(self._h, int(mode)), "wpccc_basis_set_schur_update")

    def set_wait_limit(self, polls: int) -> None:
        """Polls of every mbarrier wait in the tensor-core kernels before it gives up (ETIMEOUT); default 2^20."""
        _check(_lib.wpccc_basis_set_wait_limit(self._h, int(polls)), "wpccc_basis_set_wait_limit")

    def profile_enable(self, on: bool = True) -> None:
        """Reset the per-kernel counters; with on=True time every launch with CUDA events."""
        _check(_lib.wpccc_profile_enable(self._h, int(bool(on))), "wpccc_profile_enable")

    def profile_read(self) -> dict:
        """{category: (milliseconds, launches)} accumulated since profile_enable."""
        ms = (C.c_double * len(PROF_CATEGORIES))()
        n = (C.c_longlong * len(PROF_CATEGORIES))()
        _check(_lib.wpccc_profile_read(self._h, ms, n), "wpccc_profile_read")
        return {k: (ms[i], n[i]) for i, k in enumerate(PROF_CATEGORIES)}

    def states(self):
        """(qn, eps): qn[i] = (centre 0/1, radial index, l, m) and eps[i] of every state (``wpccc_basis_states``)."""
        qn = np.zeros((self.N, 4), dtype=np.int32)
        eps = np.zeros(self.N, dtype=np.float64)
        _check(_lib.wpccc_basis_states(self._h, qn.ctypes.data_as(_pi), eps.ctypes.data_as(_pd)),
               "wpccc_basis_states")
        return qn, eps

    def overlap_norms(self, b, v, z, c, stream=None):
        """(c^+ S c, c^+ c) of every path's amplitudes at its position (b[p], v[p], z[p]) as a device tensor
        (n_paths, 2) (``wpccc_overlap_norms``)."""
        import torch
        b = np.atleast_1d(np.asarray(b, dtype=np.float64))
        n = b.size
        v, vp = _arr(np.broadcast_to(np.asarray(v, dtype=np.float64), b.shape), np.float64)
        z, zp = _arr(np.broadcast_to(np.asarray(z, dtype=np.float64), b.shape), np.float64)
        b, bp = _arr(b, np.float64)
        _check_amplitudes(c, n, self.N, self.device, "overlap_norms")
        out = torch.empty((n, 2), dtype=torch.float64, device=c.device)
        _check(_lib.wpccc_overlap_norms(self._h, n, bp, vp, zp, _ptr(c), _ptr(out), _stream(stream)),
               "wpccc_overlap_norms")
        return out

    def matrix_elements(self, b: float, v: float, z, S=None, H=None, stream=None):
        """S, H at the positions z (column-major storage tensors of shape (nz, N, N))."""
        import torch
        z, zp = _arr(np.atleast_1d(z), np.float64)
        dev = torch.device("cuda", self.device)
        if S is None:
            S = torch.empty((z.size, self.N, self.N), dtype=torch.complex128, device=dev)
        if H is None:
            H = torch.empty((z.size, self.N, self.N), dtype=torch.complex128, device=dev)
        _check_matrices(S, H, z.size, self.N, self.device, "matrix_elements")
        _check(_lib.wpccc_matrix_elements(self._h, float(b), float(v), int(z.size), zp, _ptr(S), _ptr(H),
                                          _stream(stream)), "wpccc_matrix_elements")
        return S, H

    def matrix_elements_precision(self, b: float, v: float, z, precision_mode: int, S=None, H=None, stream=None):
        """S, H with the element arithmetic of a precision form (0 FP64, 1 FP32 contraction, 3 tensor-core
        contraction at FP32 level, 4 tensor-core contraction to FP64 accuracy), returned in FP64
        (``wpccc_matrix_elements_precision``)."""
        import torch
        z, zp = _arr(np.atleast_1d(z), np.float64)
        dev = torch.device("cuda", self.device)
        if S is None:
            S = torch.empty((z.size, self.N, self.N), dtype=torch.complex128, device=dev)
        if H is None:
            H = torch.empty((z.size, self.N, self.N), dtype=torch.complex128, device=dev)
        _check_matrices(S, H, z.size, self.N, self.device, "matrix_elements_precision")
        _check(_lib.wpccc_matrix_elements_precision(self._h, float(b), float(v), int(z.size), zp, _ptr(S), _ptr(H),
                                                    int(precision_mode), _stream(stream)),
               "wpccc_matrix_elements_precision")
        return S, H

    def matrix_elements_noalloc(self, b: float, v: float, z, S, H, stream=None):
        """Same as matrix_elements into caller-owned S, H, but the library allocates no device memory:
        its scratch is a fixed 64 MiB array shared by every call on the device (serialise calls)."""
        z, zp = _arr(np.atleast_1d(z), np.float64)
        _check_matrices(S, H, z.size, self.N, self.device, "matrix_elements_noalloc")
        _check(_lib.wpccc_matrix_elements_noalloc(self._h, float(b), float(v), int(z.size), zp, _ptr(S), _ptr(H),
                                                  _stream(stream)), "wpccc_matrix_elements_noalloc")
        return S, H

    def propagate(self, b, v, zgrids, c=None, precision_mode: int = 0, batch_mode: int = 0, stream=None):
        """Amplitudes at the end of each path (``wpccc_propagate``); `c` (n_paths, N) complex128 on the
        device is advanced in place (default: Algorithm 1's initial state)."""
        import torch
        keep = []
        pd = _paths_desc(b, v, zgrids, keep)
        if c is None:
            c = torch.zeros((pd.n_paths, self.N), dtype=torch.complex128, device=torch.device("cuda", self.device))
            c[:, 0] = 1.0
        _check_amplitudes(c, pd.n_paths, self.N, self.device, "propagate")
        _check(_lib.wpccc_propagate(self._h, C.byref(pd), int(precision_mode), int(batch_mode), _ptr(c),
                                    _stream(stream)), "wpccc_propagate")
        return c

    def propagate_adjoint(self, b, v, zgrids, g, checkpoint_every: int = 50, c=None, stream=None):
        """Observables P[p, o] = sum_i g[o, i] |c_i|^2 at the end of each path and their derivatives
        grad[p, o, k] with respect to the basis parameters (``wpccc_propagate_adjoint``; needs the basis
        tangents).  Returns (c, P, grad) as device tensors; `c` is advanced in place."""
        import torch
        keep = []
        pd = _paths_desc(b, v, zgrids, keep)
        n_paths = pd.n_paths
        dev = torch.device("cuda", self.device)
        if c is None:
            c = torch.zeros((n_paths, self.N), dtype=torch.complex128, device=dev)
            c[:, 0] = 1.0
        _check_amplitudes(c, n_paths, self.N, self.device, "propagate_adjoint")
        g, gp = _arr(np.atleast_2d(g), np.float64)
        if g.ndim != 2 or g.shape[1] != self.N:
            raise ValueError(f"observable weights must have shape (n_obs, {self.N})")
        n_obs = int(g.shape[0])
        P = torch.empty((n_paths, n_obs), dtype=torch.float64, device=dev)
        grad = torch.empty((n_paths, n_obs, max(1, self.n_par)), dtype=torch.float64, device=dev)
        _check(_lib.wpccc_propagate_adjoint(self._h, C.byref(pd), n_obs, gp, int(checkpoint_every), _ptr(c), _ptr(P),
                                            _ptr(grad), _stream(stream)), "wpccc_propagate_adjoint")
        return c, P, grad


def _paths_desc(b, v, zgrids, keep):
    b = np.atleast_1d(np.asarray(b, dtype=np.float64))
    v = np.broadcast_to(np.asarray(v, dtype=np.float64), b.shape)
    if isinstance(zgrids, np.ndarray) and zgrids.ndim == 1:
        zgrids = [zgrids] * b.size
    nz = np.array([len(zg) for zg in zgrids], dtype=np.int32)
    zc = np.concatenate([np.asarray(zg, dtype=np.float64) for zg in zgrids])
    arrs = [_arr(b, np.float64), _arr(v, np.float64), _arr(nz, np.int32), _arr(zc, np.float64)]
    keep.extend(a for a, _ in arrs)
    return _PathsDesc(n_paths=int(b.size), b=arrs[0][1], v=arrs[1][1], n_z=arrs[2][1], z=arrs[3][1])


class Batch:
    """Several (basis, paths) sets propagated together by one CUDA graph launch (``wpccc_batch_*``).

    `sets` is a list of (Basis, b, v, zgrids); `c` a list of (n_paths_k, N_k) complex128 device tensors,
    advanced in place at every launch (keep them alive while the batch exists)."""

    def __init__(self, sets, c, precision_mode: int = 0, autotune: bool = True):
        keep = []
        n = len(sets)
        if len(c) != n:
            raise ValueError(f"Batch: {n} sets but {len(c)} amplitude tensors")
        for (g, b, _, _), t in zip(sets, c):
            _check_amplitudes(t, int(np.atleast_1d(b).size), g.N, g.device, "Batch")
        descs = (_PathsDesc * n)(*[_paths_desc(b, v, zg, keep) for (_, b, v, zg) in sets])
        handles = (C.c_void_p * n)(*[g._h.value for (g, _, _, _) in sets])
        cptrs = (C.c_void_p * n)(*[t.data_ptr() for t in c])
        h = C.c_void_p()
        _check(_lib.wpccc_batch_create(n, handles, descs, int(precision_mode), cptrs, int(bool(autotune)),
                                       C.byref(h)), "wpccc_batch_create")
        self._h = h
        self.n_sets = n
        self.c = list(c)
        self._bases = [g for (g, _, _, _) in sets]

    def launch(self, stream=None) -> None:
        _check(_lib.wpccc_batch_launch(self._h, _stream(stream)), "wpccc_batch_launch")

    def status(self, stream=None) -> None:
        _check(_lib.wpccc_batch_status(self._h, _stream(stream)), "wpccc_batch_status")

    def info(self):
        """(RK4 steps per chunk, autotuner ms per step) for every set."""
        cs = np.zeros(self.n_sets, dtype=np.int32)
        ms = np.zeros(self.n_sets, dtype=np.float64)
        _check(_lib.wpccc_batch_info(self._h, cs.ctypes.data_as(_pi), ms.ctypes.data_as(_pd)), "wpccc_batch_info")
        return cs, ms

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.wpccc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(S, H, precision_mode: int = 0, stream=None):
    """Batched S X = H in place on column-major storage tensors (batch, N, N); returns (ipiv, info)."""
    import torch
    batch, N = S.shape[0], S.shape[-1]
    ipiv = torch.empty((batch, N), dtype=torch.int32, device=S.device)
    info = torch.empty((batch,), dtype=torch.int32, device=S.device)
    _check(_lib.wpccc_solve(int(N), int(batch), _ptr(S), _ptr(H), _ptr(ipiv), _ptr(info), int(precision_mode),
                            _stream(stream)), "wpccc_solve")
    return ipiv, info


def probabilities(c, stream=None):
    """|c|^2 for a (n_paths, N) complex128 device tensor (``wpccc_probabilities``)."""
    import torch
    n_paths, N = c.shape
    P = torch.empty((n_paths, N), dtype=torch.float64, device=c.device)
    _check(_lib.wpccc_probabilities(int(n_paths), int(N), _ptr(c), _ptr(P), _stream(stream)),
           "wpccc_probabilities")
    return P


def observables_of(c, g, stream=None):
    """P[p, o] = sum_i g[o, i] |c[p, i]|^2 for a (n_paths, N) complex128 device tensor c and weights g
    (n_obs, N) (``wpccc_observables``)."""
    import torch
    n_paths, N = c.shape
    gt = torch.as_tensor(np.atleast_2d(np.asarray(g, dtype=np.float64)), device=c.device).contiguous()
    if gt.shape[1] != N:
        raise ValueError(f"observable weights must have shape (n_obs, {N})")
    n_obs = int(gt.shape[0])
    P = torch.empty((n_paths, n_obs), dtype=torch.float64, device=c.device)
    _check(_lib.wpccc_observables(int(n_paths), int(N), n_obs, _ptr(gt), _ptr(c), _ptr(P), _stream(stream)),
           "wpccc_observables")
    return P


def cross_sections(b, P, stream=None):
    """sigma_o = 2 pi int b P_o(b) db by the trapezoid rule on the (increasing) impact parameters b and the
    node b = 0, for P (n_b, n_obs) (a device tensor, or a host array copied to the current device)
    (``wpccc_cross_sections``); returns a device tensor (n_obs,)."""
    import torch
    b, bp = _arr(np.atleast_1d(b), np.float64)
    Pt = torch.as_tensor(P, dtype=torch.float64)
    if Pt.device.type != "cuda":
        Pt = Pt.cuda()
    Pt = Pt.reshape(b.size, -1).contiguous()
    n_obs = int(Pt.shape[1])
    sigma = torch.empty((n_obs,), dtype=torch.float64, device=Pt.device)
    _check(_lib.wpccc_cross_sections(int(b.size), bp, n_obs, _ptr(Pt), _ptr(sigma), _stream(stream)),
           "wpccc_cross_sections")
    return sigma


def _observables_function():
    import torch

    class Observables(torch.autograd.Function):
        """P[p, o] = sum_i g[o, i] |c_i|^2 at the end of every path as a function of the parameters theta.

        `make_basis(theta)` returns the ``wpccc_inputs`` basis (with its parameter tangents) at theta.
        The forward pass runs the adjoint propagation when theta needs a gradient (keeping the
        Jacobian dP/dtheta for the backward pass) and the plain propagation otherwise."""

        @staticmethod
        def forward(ctx, theta, make_basis, b, v, zgrids, g, checkpoint_every=50, device=0):
            th = theta.detach().cpu().numpy().astype(np.float64)
            gb = Basis(make_basis(th), device)
            try:
                if ctx.needs_input_grad[0]:
                    _, P, J = gb.propagate_adjoint(b, v, zgrids, g, checkpoint_every)
                    ctx.save_for_backward(J)
                else:
                    c = gb.propagate(b, v, zgrids)
                    P = observables_of(c, g)
            finally:
                gb.close()
            ctx.theta_device = theta.device
            return P

        @staticmethod
        def backward(ctx, grad_out):
            (J,) = ctx.saved_tensors
            gt = torch.einsum("po,pok->k", grad_out.to(J.dtype), J)
            return (gt.to(ctx.theta_device),) + (None,) * 7

    return Observables


def observables(theta, make_basis, b, v, zgrids, g, checkpoint_every: int = 50, device: int = 0):
    """Differentiable end-of-path observables (see ``_observables_function``): a torch tensor of shape
    (n_paths, n_obs); ``.backward()`` gives d/dtheta through the adjoint of the propagation."""
    return _observables_function().apply(theta, make_basis, b, v, zgrids, g, checkpoint_every, device)
