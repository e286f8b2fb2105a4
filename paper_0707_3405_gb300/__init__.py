"""GB300 (sm_103a) block LOBPCG plane-wave eigensolver -- Python binding.

A thin ctypes layer over the C ABI in ``include/lobpcg_gb300.h`` and
``include/lobpcg_gb300_kernels.h``.  It only marshals arguments: every step
of the computation runs in the CUDA library ``_lib/liblobpcg_gb300.so``.
PyTorch is used for device memory and CUDA streams.

Array conventions: a block of nb bands of one k-point is a tensor of shape
``(nb, npw)`` (row b = band b), which is the library's column-major
npw x nb layout.  Projectors are given as ``(npw, nproj)`` numpy arrays.

There is no fallback: if the library has not been built, importing the
binding succeeds but every call raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblobpcg_gb300.so")

OK, NOT_CONVERGED = 0, 1
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BREAKDOWN, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
C128, C64, C128_DF32, C128_TC = 0, 1, 2, 3
FP64, MIXED = 0, 1

EXPORTED = (
    "lobpcg_default_options", "lobpcg_create", "lobpcg_set_projectors", "lobpcg_set_stream",
    "lobpcg_set_options", "lobpcg_npw", "lobpcg_gvectors", "lobpcg_apply_H", "lobpcg_solve",
    "lobpcg_last_error", "lobpcg_destroy", "lobpcg_struct_sizes", "lobpcg_launch_count", "lobpcg_apply_local_noalloc",
    "lobpcg_density", "lobpcg_solve_pcg",
    "lobpcg_k_gemm_cn", "lobpcg_k_gram_lower", "lobpcg_k_gemm_nn", "lobpcg_k_rayleigh_ritz", "lobpcg_k_rayleigh_ritz_df32", "lobpcg_k_rayleigh_ritz32", "lobpcg_k_heev",
    "lobpcg_k_set_gemm_mode", "lobpcg_k_set_spin_limit", "lobpcg_k_check_timeouts", "lobpcg_k_last_error",
)


class Cell(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("N", ctypes.c_int), ("ecut", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int), ("nline", ctypes.c_int), ("max_sweeps", ctypes.c_int),
                ("precision", ctypes.c_int), ("gemm_split", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("autotune", ctypes.c_int), ("tol", ctypes.c_double), ("mem_cap", ctypes.c_longlong),
                ("timing", ctypes.c_int), ("nbuf", ctypes.c_int), ("mixed_switch", ctypes.c_double),
                ("mixed_early", ctypes.c_double), ("fp64_gemm", ctypes.c_int), ("gamma_real", ctypes.c_int)]


PHASES = ("fft", "nonlocal", "gram", "constraint", "rr", "update")
NPH = len(PHASES)


class Stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("restarts", ctypes.c_int), ("max_resid", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("band_applies_fp64", ctypes.c_longlong), ("band_applies_fp32", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong),
                ("ph_ms", ctypes.c_double * NPH), ("ph_flops", ctypes.c_double * NPH),
                ("ph_bytes", ctypes.c_double * NPH), ("ph_calls", ctypes.c_longlong * NPH),
                ("ph_fp64_flops", ctypes.c_double * NPH),
                ("block_visits_fp32", ctypes.c_longlong), ("block_visits_fp64", ctypes.c_longlong),
                ("ph_ms_fp64", ctypes.c_double * NPH), ("ph_bytes_fp64", ctypes.c_double * NPH),
                ("block_visits_settled", ctypes.c_longlong), ("ms_autotune", ctypes.c_double)]

    def as_dict(self) -> dict:
        out = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            out[f] = {p: v[i] for i, p in enumerate(PHASES)} if f.startswith("ph_") else v
        return out


class LobpcgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lobpcg error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return LIB_PATH


def load() -> ctypes.CDLL:
    """Load the CUDA library; raises RuntimeError when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "lobpcg_default_options": (i, [ctypes.POINTER(Options)]),
        "lobpcg_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(Cell), i, vp, vp, i, vp, vp, ctypes.POINTER(Options), vp]),
        "lobpcg_set_projectors": (i, [vp, i, vp]),
        "lobpcg_set_stream": (i, [vp, vp]),
        "lobpcg_set_options": (i, [vp, ctypes.POINTER(Options)]),
        "lobpcg_npw": (i, [vp, i]),
        "lobpcg_gvectors": (i, [vp, i, vp]),
        "lobpcg_apply_H": (i, [vp, i, vp, vp, i, i]),
        "lobpcg_solve": (i, [vp, i, vp, vp, vp, ctypes.POINTER(Stats)]),
        "lobpcg_last_error": (ctypes.c_char_p, [vp]),
        "lobpcg_destroy": (None, [vp]),
        "lobpcg_struct_sizes": (i, [ctypes.POINTER(ctypes.c_int64)] * 3),
        "lobpcg_launch_count": (ctypes.c_longlong, []),
        "lobpcg_apply_local_noalloc": (i, [vp, i, vp, vp, i, i]),
        "lobpcg_density": (i, [vp, i, vp, i, vp, vp, i]),
        "lobpcg_solve_pcg": (i, [vp, i, vp, vp, vp, ctypes.POINTER(Stats)]),
        "lobpcg_k_gemm_cn": (i, [i, i, i, i, d, vp, i, vp, i, d, vp, i, vp]),
        "lobpcg_k_gram_lower": (i, [i, i, i, vp, i, vp, i, vp, i, vp]),
        "lobpcg_k_gemm_nn": (i, [i, i, i, i, d, vp, i, vp, i, d, vp, i, vp, i, vp]),
        "lobpcg_k_rayleigh_ritz": (i, [i, i, vp, vp, d, vp, vp, vp, vp]),
        "lobpcg_k_rayleigh_ritz_df32": (i, [i, i, vp, vp, d, vp, vp, vp, vp]),
        "lobpcg_k_rayleigh_ritz32": (i, [i, i, vp, vp, d, vp, vp, vp, vp]),
        "lobpcg_k_heev": (i, [i, vp, vp, vp, vp]),
        "lobpcg_k_set_gemm_mode": (i, [i]),
        "lobpcg_k_set_spin_limit": (i, [ll]),
        "lobpcg_k_check_timeouts": (i, []),
        "lobpcg_k_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    # the structures above must match the library's layout exactly (the library writes them)
    sizes = [ctypes.c_int64() for _ in range(3)]
    lib.lobpcg_struct_sizes(*[ctypes.byref(x) for x in sizes])
    mine = (ctypes.sizeof(Cell), ctypes.sizeof(Options), ctypes.sizeof(Stats))
    if tuple(x.value for x in sizes) != mine:
        raise RuntimeError(f"binding and library disagree on struct sizes (cell, options, stats): "
                           f"{mine} here, {tuple(x.value for x in sizes)} in {LIB_PATH}")
    _lib = lib
    return lib


def _ptr(t) -> int:
    """Device or host address of a torch tensor or numpy array."""
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _stream_handle(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dev_mats(*ops):
    """Raise unless every ``(name, tensor, dtype, shape)`` names a contiguous CUDA tensor of that
    dtype and shape: the dense building blocks take device pointers with sizes derived from the
    other operands.  Types and shapes are checked for all operands before residency."""
    import torch
    for name, t, dtype, shape in ops:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, not {t.dtype}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}, not {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    for name, t, _, _ in ops:
        if not t.is_cuda:
            raise TypeError(f"{name} must be on a CUDA device")


def _band_block(name: str, x, npw: int):
    """Raise unless ``x`` (numpy array or torch tensor, host or device) is a C-contiguous
    complex128 (rows, npw) block."""
    if isinstance(x, np.ndarray):
        ok_type, contig = x.dtype == np.complex128, x.flags.c_contiguous
    elif hasattr(x, "is_contiguous"):
        import torch
        ok_type, contig = x.dtype == torch.complex128, x.is_contiguous()
    else:
        raise TypeError(f"{name} must be a numpy array or a torch tensor")
    if not ok_type:
        raise TypeError(f"{name} must be complex128")
    if x.ndim != 2 or x.shape[1] != npw:
        raise ValueError(f"{name} must have shape (rows, {npw}), not {tuple(x.shape)}")
    if not contig:
        raise ValueError(f"{name} must be contiguous")


def default_options() -> Options:
    o = Options()
    _check(load().lobpcg_default_options(ctypes.byref(o)), None)
    return o


def _check(rc: int, handle, kernels: bool = False) -> int:
    if rc < 0:
        lib = load()
        if kernels:
            msg = lib.lobpcg_k_last_error()
        else:
            msg = lib.lobpcg_last_error(handle)
        raise LobpcgError(rc, (msg or b"").decode(errors="replace"))
    return rc


@dataclass
class SolveResult:
    eig: np.ndarray      # (nk, M)
    resid: np.ndarray    # (nk, M)
    status: int
    stats: dict


class Solver:
    """One cell, its k-points, potential and projectors: ``lobpcg_create``.

    ``kpts`` (nk, 3) reduced; ``vloc`` (N, N, N) float64 [x][y][z];
    ``proj_E`` (nproj,) KB energies; ``beta`` optional callable
    ``beta(miller (npw,3) int, k_index) -> (npw, nproj) complex128`` giving the
    projectors in the library's plane-wave order.
    """

    def __init__(self, a: float, N: int, ecut: float, kpts, vloc, proj_E=None, beta=None,
                 block_size: int = 64, nline: int = 4, max_sweeps: int = 100, precision: str = "fp64",
                 tol: float = 1e-8, mem_cap: int = 0, timing: bool = False, nbuf: int = 0,
                 mixed_switch: float | None = None, mixed_early: float | None = None, stream=None,
                 fp64_gemm: int = 0, use_graph: bool = False, autotune: bool = False, gamma_real: bool = False):
        lib = load()
        self._lib = lib
        self.handle = ctypes.c_void_p()
        kp = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
        v = np.ascontiguousarray(np.asarray(vloc, dtype=np.float64))
        if v.shape != (N, N, N):
            raise ValueError("vloc must have shape (N, N, N)")
        E = np.ascontiguousarray(np.zeros(0) if proj_E is None else np.asarray(proj_E, dtype=np.float64))
        self.nproj = int(E.shape[0])
        self.nk = int(kp.shape[0])
        opt = self._options(block_size, nline, max_sweeps, precision, tol, mem_cap, timing, nbuf, mixed_switch,
                            mixed_early, fp64_gemm, use_graph, autotune, gamma_real)
        cell = Cell(a, N, ecut)
        self._stream = stream
        rc = lib.lobpcg_create(ctypes.byref(self.handle), ctypes.byref(cell), self.nk, kp.ctypes.data,
                               v.ctypes.data, self.nproj, E.ctypes.data if self.nproj else None, None,
                               ctypes.byref(opt), _stream_handle(stream))
        if rc < 0:
            raise LobpcgError(rc, (lib.lobpcg_last_error(None) or b"").decode(errors="replace"))
        self.a, self.N, self.ecut = a, N, ecut
        self.kpts = kp
        if self.nproj and beta is not None:
            for k in range(self.nk):
                self.set_projectors(k, beta(self.gvectors(k), k))

    @staticmethod
    def _options(block_size, nline, max_sweeps, precision, tol, mem_cap, timing=False, nbuf=0,
                 mixed_switch=None, mixed_early=None, fp64_gemm=0, use_graph=False, autotune=False,
                 gamma_real=False) -> Options:
        o = default_options()
        o.block_size, o.nline, o.max_sweeps = block_size, nline, max_sweeps
        o.precision = {"fp64": FP64, "mixed": MIXED}[precision]
        o.tol = tol
        o.mem_cap = mem_cap
        o.timing = 1 if timing else 0
        o.nbuf = nbuf
        if mixed_switch is not None:
            o.mixed_switch = mixed_switch
        if mixed_early is not None:
            o.mixed_early = mixed_early
        o.fp64_gemm = fp64_gemm
        o.use_graph = 1 if use_graph else 0
        o.autotune = 1 if autotune else 0
        o.gamma_real = 1 if gamma_real else 0
        return o

    def set_options(self, block_size=64, nline=4, max_sweeps=100, precision="fp64", tol=1e-8, mem_cap=0,
                    timing=False, nbuf=0, mixed_switch=None, mixed_early=None, fp64_gemm=0, use_graph=False,
                    autotune=False, gamma_real=False):
        o = self._options(block_size, nline, max_sweeps, precision, tol, mem_cap, timing, nbuf, mixed_switch,
                          mixed_early, fp64_gemm, use_graph, autotune, gamma_real)
        _check(self._lib.lobpcg_set_options(self.handle, ctypes.byref(o)), self.handle)

    def set_stream(self, stream):
        self._stream = stream
        _check(self._lib.lobpcg_set_stream(self.handle, _stream_handle(stream)), self.handle)

    def npw(self, k: int = 0) -> int:
        return _check(self._lib.lobpcg_npw(self.handle, k), self.handle)

    def gvectors(self, k: int = 0) -> np.ndarray:
        out = np.empty((self.npw(k), 3), dtype=np.int32)
        _check(self._lib.lobpcg_gvectors(self.handle, k, out.ctypes.data), self.handle)
        return out

    def set_projectors(self, k: int, beta: np.ndarray):
        b = np.asarray(beta, dtype=np.complex128)
        if b.shape != (self.npw(k), self.nproj):
            raise ValueError("beta must have shape (npw_k, nproj)")
        colmajor = np.ascontiguousarray(b.T)
        _check(self._lib.lobpcg_set_projectors(self.handle, k, colmajor.ctypes.data), self.handle)

    def apply_H(self, k: int, X, Y=None, df32: bool = False, tc: bool = False):
        """Y = H X for a (nb, npw) block: torch CUDA tensor (asynchronous on the
        handle's stream) or numpy array (staged, synchronous).  complex128 runs
        in FP64 (or double-FP32 with df32=True, or double-FP32 FFT with the KB
        products on the tensor cores with tc=True), complex64 in FP32."""
        import torch
        if isinstance(X, np.ndarray):
            prec = C128 if X.dtype == np.complex128 else C64
            if X.dtype not in (np.complex128, np.complex64):
                raise TypeError("X must be complex64 or complex128")
            X = np.ascontiguousarray(X)
            if Y is None:
                Y = np.empty_like(X)
            elif not (isinstance(Y, np.ndarray) and Y.dtype == X.dtype and Y.shape == X.shape
                      and Y.flags.c_contiguous):
                raise TypeError("Y must be a contiguous numpy array with the shape and dtype of X")
        else:
            prec = C128 if X.dtype == torch.complex128 else C64
            if X.dtype not in (torch.complex128, torch.complex64):
                raise TypeError("X must be complex64 or complex128")
            if not X.is_contiguous():
                raise ValueError("X must be contiguous")
            if Y is None:
                Y = torch.empty_like(X)
            elif not (isinstance(Y, torch.Tensor) and Y.dtype == X.dtype and Y.shape == X.shape
                      and Y.device == X.device and Y.is_contiguous()):
                raise TypeError("Y must be a contiguous tensor with the shape, dtype and device of X")
        if X.ndim != 2:
            raise ValueError("X must be an (nb, npw_k) block")
        nb = 0 if X.shape[0] == 0 else int(X.shape[0])
        if nb and X.shape[-1] != self.npw(k):
            raise ValueError("X must have shape (nb, npw_k)")
        if df32 or tc:
            if prec != C128:
                raise ValueError("df32 / tc need complex128 vectors")
            prec = C128_TC if tc else C128_DF32
        _check(self._lib.lobpcg_apply_H(self.handle, k, _ptr(X), _ptr(Y), nb, prec), self.handle)
        return Y

    def apply_local_noalloc(self, k: int, X, Y):
        """Y = (T + V_loc) X without any device allocation (the library's fixed
        32 MiB scratch array holds the FFT half-box).  X and Y are (nb, npw)
        CUDA tensors, complex128 or complex64."""
        import torch
        if X.dtype not in (torch.complex128, torch.complex64):
            raise TypeError("X must be complex64 or complex128")
        if not (isinstance(Y, torch.Tensor) and Y.dtype == X.dtype and tuple(Y.shape) == tuple(X.shape)):
            raise TypeError("Y must be a tensor with the shape and dtype of X")
        if X.dim() != 2 or not X.is_contiguous() or not Y.is_contiguous():
            raise ValueError("X and Y must be contiguous (nb, npw_k) blocks")
        if X.shape[0] and X.shape[1] != self.npw(k):
            raise ValueError("X must have shape (nb, npw_k)")
        prec = C128 if X.dtype == torch.complex128 else C64
        rc = self._lib.lobpcg_apply_local_noalloc(self.handle, k, _ptr(X), _ptr(Y), int(X.shape[0]), prec)
        if rc < 0:
            raise LobpcgError(rc, (self._lib.lobpcg_last_error(None) or b"").decode(errors="replace"))
        return Y

    def density(self, k: int, X, f, rho=None, df32: bool = False):
        """rho += sum_b f_b |psi_b(r)|^2 on the N^3 grid ([x][y][z], float64 CUDA tensor,
        created zero when None) for the (nb, npw_k) CUDA block X; complex128 runs FP64
        transforms (double-FP32 with df32=True), complex64 FP32 ones.  Returns rho."""
        import torch
        if X.dtype not in (torch.complex128, torch.complex64):
            raise TypeError("X must be complex64 or complex128")
        if X.dim() != 2 or not X.is_contiguous() or (X.shape[0] and X.shape[1] != self.npw(k)):
            raise ValueError("X must be a contiguous (nb, npw_k) block")
        fh = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
        if fh.shape[0] != X.shape[0]:
            raise ValueError("one occupation per band is needed")
        if rho is None:
            rho = torch.zeros((self.N, self.N, self.N), dtype=torch.float64, device=X.device)
        if rho.dtype != torch.float64 or tuple(rho.shape) != (self.N,) * 3 or not rho.is_contiguous():
            raise ValueError("rho must be a contiguous float64 (N, N, N) tensor")
        prec = C64 if X.dtype == torch.complex64 else (C128_DF32 if df32 else C128)
        _check(self._lib.lobpcg_density(self.handle, k, _ptr(X), int(X.shape[0]), fh.ctypes.data, _ptr(rho), prec),
               self.handle)
        return rho

    def solve(self, X, nbands: int | None = None, method: str = "lobpcg") -> SolveResult:
        """Lowest eigenpairs; ``X`` is a list (one per k-point) of (M, npw_k)
        complex128 CUDA tensors holding start vectors, overwritten by the
        eigenvectors.  method = "lobpcg" (block LOBPCG, Algorithm 1) or "pcg"
        (band-by-band PCG, the comparison method of Sec. 3.3)."""
        if not isinstance(X, (list, tuple)):
            X = [X]
        if len(X) != self.nk:
            raise ValueError("one start block per k-point is needed")
        for k, x in enumerate(X):
            _band_block(f"X[{k}]", x, self.npw(k))
        M = int(X[0].shape[0]) if nbands is None else int(nbands)
        if any(x.shape[0] < M for x in X):
            raise ValueError(f"every start block needs at least nbands = {M} rows")
        ptrs = (ctypes.c_void_p * self.nk)(*[ctypes.c_void_p(_ptr(x)) for x in X])
        eig = np.zeros((self.nk, M))
        res = np.zeros((self.nk, M))
        st = Stats()
        fn = {"lobpcg": self._lib.lobpcg_solve, "pcg": self._lib.lobpcg_solve_pcg}[method]
        rc = _check(fn(self.handle, M, ptrs, eig.ctypes.data, res.ctypes.data, ctypes.byref(st)), self.handle)
        return SolveResult(eig, res, rc, st.as_dict())

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self._lib.lobpcg_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load().lobpcg_launch_count())


# ---------------------------------------------------------------- dense building blocks
def set_gemm_mode(mode: int):
    """Complex64 GEMM engine of the calling thread: 0 or 2 = tensor cores (3xTF32) for long
    reductions and tall products, 3 = CUDA cores only."""
    _check(load().lobpcg_k_set_gemm_mode(int(mode)), None, kernels=True)


def set_spin_limit(polls: int):
    """Poll limit of the tensor-core GEMMs' ring waits (< 0: default); for tests of the
    timeout path."""
    _check(load().lobpcg_k_set_spin_limit(int(polls)), None, kernels=True)


def check_timeouts():
    """Synchronise; raise LobpcgError(ERR_TIMEOUT) if a tensor-core GEMM gave up waiting."""
    _check(load().lobpcg_k_check_timeouts(), None, kernels=True)


def _prec128(dtype, df32, tc):
    import torch
    if dtype not in (torch.complex128, torch.complex64):
        raise TypeError("operands must be complex64 or complex128")
    prec = C128 if dtype == torch.complex128 else C64
    if df32 or tc:
        if prec != C128:
            raise ValueError("df32 / tc need complex128 operands")
        prec = C128_TC if tc else C128_DF32
    return prec


def gemm_cn(A, B, alpha=1.0, beta=0.0, C=None, stream=None, df32=False, tc=False):
    """C = alpha A^H B + beta C for torch CUDA tensors given as (cols, rows) row-major
    (i.e. column-major matrices): A is (m, K), B is (n, K), C is (n, m).  df32=True
    (complex128 only) runs the double-FP32 engine instead of FP64 arithmetic, tc=True
    the FP64-class tensor-core engine (exact BF16 digit slices)."""
    import torch
    lib = load()
    prec = _prec128(A.dtype, df32, tc)
    if A.dim() != 2 or B.dim() != 2:
        raise ValueError("A and B must be matrices")
    m, K = A.shape
    n = B.shape[0]
    if C is None:
        C = torch.zeros((n, m), dtype=A.dtype, device=A.device)
    _dev_mats(("A", A, A.dtype, (m, K)), ("B", B, A.dtype, (n, K)), ("C", C, A.dtype, (n, m)))
    _check(lib.lobpcg_k_gemm_cn(prec, m, n, K, alpha, _ptr(A), K, _ptr(B), K, beta, _ptr(C), m,
                                _stream_handle(stream)), None, kernels=True)
    return C


def gram_lower(A, B, C=None, stream=None, df32=False, tc=False):
    """Lower triangle of C = A^H B (complex128), column-major as in gemm_cn: A and B are
    (n, K), C is (n, n).  Tiles of C strictly above the diagonal are left untouched.
    df32=True runs the double-FP32 engine instead of FP64 arithmetic, tc=True the
    tensor-core engine (which writes only the entries i >= j)."""
    import torch
    lib = load()
    n, K = A.shape
    if A.dtype != torch.complex128 or B.dtype != torch.complex128 or B.shape != A.shape:
        raise ValueError("gram_lower: A and B must be complex128 of the same shape")
    if C is None:
        C = torch.zeros((n, n), dtype=A.dtype, device=A.device)
    _dev_mats(("A", A, torch.complex128, (n, K)), ("B", B, torch.complex128, (n, K)),
              ("C", C, torch.complex128, (n, n)))
    _check(lib.lobpcg_k_gram_lower(C128_TC if tc else (C128_DF32 if df32 else C128), n, K, _ptr(A), K, _ptr(B), K, _ptr(C), n,
                                   _stream_handle(stream)), None, kernels=True)
    return C


def gemm_nn(A, B, alpha=1.0, beta=0.0, C=None, D=None, stream=None, df32=False, tc=False):
    """D = alpha A B + beta C, column-major stored as transposed torch tensors:
    A is (k, M), B is (n, k), C and D are (n, M).  df32 and tc as in gemm_cn."""
    import torch
    lib = load()
    prec = _prec128(A.dtype, df32, tc)
    if A.dim() != 2 or B.dim() != 2:
        raise ValueError("A and B must be matrices")
    k, M = A.shape
    n = B.shape[0]
    if D is None:
        D = torch.empty((n, M), dtype=A.dtype, device=A.device)
    ops = [("A", A, A.dtype, (k, M)), ("B", B, A.dtype, (n, k)), ("D", D, A.dtype, (n, M))]
    _dev_mats(*(ops + ([("C", C, A.dtype, (n, M))] if C is not None else [])))
    _check(lib.lobpcg_k_gemm_nn(prec, M, n, k, alpha, _ptr(A), M, _ptr(B), k, beta,
                                _ptr(C) if C is not None else None, M, _ptr(D), M, _stream_handle(stream)),
           None, kernels=True)
    return D


def rayleigh_ritz(S, A, m, drop_tol=1e-12, stream=None, df32=False):
    """Lowest m pairs of A c = theta S c (n x n complex128 CUDA tensors, column-major
    i.e. pass the transpose of a numpy matrix).  Returns (theta (m,), C (m, n) whose
    row j is column j of the coefficient matrix, ndropped).  df32=True runs the
    FP64-unit-bound parts in double-FP32 arithmetic."""
    import torch
    lib = load()
    n = S.shape[0]
    _dev_mats(("S", S, torch.complex128, (n, n)), ("A", A, torch.complex128, (n, n)))
    theta = torch.empty(m, dtype=torch.float64, device=S.device)
    C = torch.empty((m, n), dtype=torch.complex128, device=S.device)
    nd = torch.zeros(1, dtype=torch.int32, device=S.device)
    fn = lib.lobpcg_k_rayleigh_ritz_df32 if df32 else lib.lobpcg_k_rayleigh_ritz
    _check(fn(n, m, _ptr(S), _ptr(A), drop_tol, _ptr(theta), _ptr(C), _ptr(nd), _stream_handle(stream)), None,
           kernels=True)
    return theta, C, nd


def rayleigh_ritz32(S, A, m, drop_tol=1e-3, stream=None):
    """FP32 version of rayleigh_ritz on complex64 CUDA tensors (column-major)."""
    import torch
    lib = load()
    n = S.shape[0]
    _dev_mats(("S", S, torch.complex64, (n, n)), ("A", A, torch.complex64, (n, n)))
    theta = torch.empty(m, dtype=torch.float32, device=S.device)
    C = torch.empty((m, n), dtype=torch.complex64, device=S.device)
    nd = torch.zeros(1, dtype=torch.int32, device=S.device)
    _check(lib.lobpcg_k_rayleigh_ritz32(n, m, _ptr(S), _ptr(A), drop_tol, _ptr(theta), _ptr(C), _ptr(nd),
                                        _stream_handle(stream)), None, kernels=True)
    return theta, C, nd


def heev(A, stream=None):
    """Eigen-decomposition of an n x n complex128 CUDA tensor (column-major; lower
    triangle used).  Returns (w (n,), V (n, n) whose row j is eigenvector j)."""
    import torch
    lib = load()
    n = A.shape[0]
    _dev_mats(("A", A, torch.complex128, (n, n)))
    w = torch.empty(n, dtype=torch.float64, device=A.device)
    V = torch.empty((n, n), dtype=torch.complex128, device=A.device)
    _check(lib.lobpcg_k_heev(n, _ptr(A), _ptr(w), _ptr(V), _stream_handle(stream)), None, kernels=True)
    return w, V
