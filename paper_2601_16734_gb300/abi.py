"""Thin ctypes binding of libseemps_gb300.so.

Argument marshalling only: every function forwards device pointers of torch
tensors (float64, contiguous, on the context's device) to the C entry point
of the same name and raises SeempsError on a non-zero status.  Torch supplies
device memory and the stream; all arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

from . import _build

_LIB = None

OK = 0
FP64, BF16X3, FP64X2 = 0, 1, 2
LEFT, RIGHT = 0, 1
TRUNC_WEIGHT, TRUNC_RELATIVE = 0, 1
ABSORB_RIGHT, ABSORB_LEFT = 0, 1
PRECOND_NONE, PRECOND_JACOBI, PRECOND_MLP = 0, 1, 2
MODE_EIG, MODE_SOLVE, MODE_SIMPLIFY, MODE_TDVP, MODE_APPLY = 0, 1, 2, 3, 4

STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "CUDA", 3: "WORKSPACE", 4: "NOT_CONVERGED",
                5: "TIMEOUT", 6: "NUMERICAL", 7: "UNSUPPORTED"}


class SeempsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"seemps status {status} ({STATUS_NAMES.get(status, '?')}): {msg}")
        self.status = status


class Strategy(C.Structure):
    _fields_ = [("chi_max", C.c_int), ("tol", C.c_double), ("rule", C.c_int)]


class PairDims(C.Structure):
    _fields_ = [("chi_l", C.c_int), ("chi_r", C.c_int), ("d", C.c_int),
                ("D_l", C.c_int), ("D_m", C.c_int), ("D_r", C.c_int)]


class ChainC(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("d", C.c_int),
                ("D", C.POINTER(C.c_int)), ("W", C.POINTER(C.c_void_p)),
                ("A", C.POINTER(C.c_void_p)), ("chi", C.POINTER(C.c_int)),
                ("Lenv", C.POINTER(C.c_void_p)), ("Renv", C.POINTER(C.c_void_p)),
                ("B", C.POINTER(C.c_void_p)), ("chib", C.POINTER(C.c_int)),
                ("Fenv", C.POINTER(C.c_void_p)), ("Genv", C.POINTER(C.c_void_p))]


class SweepParams(C.Structure):
    _fields_ = [("mode", C.c_int), ("n_sweeps", C.c_int), ("refine_sweeps", C.c_int),
                ("precision", C.c_int), ("krylov_dim", C.c_int), ("breakdown_tol", C.c_double),
                ("strategy", Strategy), ("canonicalize", C.c_int), ("pcg_rtol", C.c_double),
                ("pcg_maxiter", C.c_int), ("precond", C.c_int), ("mlp", C.c_void_p),
                ("tdvp_dt", C.c_double)]


class SweepReport(C.Structure):
    _fields_ = [("energy", C.c_double), ("max_discarded", C.c_double),
                ("error_bound", C.c_double), ("local_iters", C.c_longlong),
                ("seconds", C.c_double), ("half_sweeps", C.c_int),
                ("half_sweep_energy", C.POINTER(C.c_double)),
                ("half_sweep_max_rank", C.POINTER(C.c_int))]


class CgsProblem(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("d", C.c_int), ("D", C.POINTER(C.c_int)), ("W", C.POINTER(C.c_void_p)),
                ("chib", C.POINTER(C.c_int)), ("B", C.POINTER(C.c_void_p)), ("chix", C.POINTER(C.c_int)),
                ("X", C.POINTER(C.c_void_p)), ("work", C.c_void_p), ("work_bytes", C.c_size_t)]


class CgsParams(C.Structure):
    _fields_ = [("strategy", Strategy), ("n_sweeps", C.c_int), ("precision", C.c_int), ("maxiter", C.c_int),
                ("rtol", C.c_double)]


class CgsReport(C.Structure):
    _fields_ = [("iterations", C.c_int), ("residual", C.c_double), ("norm_b", C.c_double),
                ("seconds", C.c_double), ("residual_history", C.POINTER(C.c_double))]


class MlpDataset(C.Structure):
    _fields_ = [("n_systems", C.c_int), ("dims", C.POINTER(PairDims)), ("L", C.POINTER(C.c_void_p)),
                ("W1", C.POINTER(C.c_void_p)), ("W2", C.POINTER(C.c_void_p)), ("R", C.POINTER(C.c_void_p)),
                ("b", C.POINTER(C.c_void_p)), ("xstar", C.POINTER(C.c_void_p)), ("site", C.POINTER(C.c_int)),
                ("n_sites", C.POINTER(C.c_int))]


class MlpTrainParams(C.Structure):
    _fields_ = [("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float)]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_SIGS = {
    "seemps_cgs_work_bytes": [_I, _I, _I, _I, _I, C.POINTER(C.c_size_t)],
    "seemps_cgs_solve": [_P, C.POINTER(CgsProblem), C.POINTER(CgsParams), C.POINTER(CgsReport)],
    "seemps_workspace_bytes": [_I, _I, _I, _I, _I, C.POINTER(C.c_size_t)],
    "seemps_create": [C.POINTER(_P), _I, _P, _P, C.c_size_t],
    "seemps_destroy": [_P],
    "seemps_set_stream": [_P, _P],
    "seemps_set_wait_limit": [_P, C.c_longlong],
    "seemps_set_fused_mixing": [_P, _I],
    "seemps_device_status": [_P, C.POINTER(_I)],
    "seemps_launch_count": [_P, C.POINTER(C.c_longlong)],
    "seemps_env_update": [_P, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _I],
    "seemps_env_update_braket": [_P, _I, _I, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _P, _I],
    "seemps_heff_apply_braket": [_P, C.POINTER(PairDims), _I, _I, _P, _P, _P, _P, _P, _P, _I],
    "seemps_env_update_linear": [_P, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P],
    "seemps_two_site": [_P, _I, _I, _I, _I, _P, _P, _P],
    "seemps_heff_apply": [_P, C.POINTER(PairDims), _P, _P, _P, _P, _P, _P, _I],
    "seemps_heff_diagonal": [_P, C.POINTER(PairDims), _P, _P, _P, _P, _P],
    "seemps_b_effective": [_P, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _P],
    "seemps_local_eig": [_P, C.POINTER(PairDims), _P, _P, _P, _P, _P, _I, _D, _I, _P, _P],
    "seemps_heff1_apply": [_P, C.POINTER(PairDims), _P, _P, _P, _P, _P, _I],
    "seemps_local_expm": [_P, C.POINTER(PairDims), _I, _P, _P, _P, _P, _P, _I, _D, _D, _I, _P, _P],
    "seemps_local_pcg": [_P, C.POINTER(PairDims), _P, _P, _P, _P, _P, _P, _I, _P, _D, _I, _I,
                         _P, _P],
    "seemps_svd_truncate": [_P, _I, _I, _P, C.POINTER(Strategy), _I, _I, _P, _P, _P, _P, _P, _I, _I],
    "seemps_truncation_rank": [_P, _I, _P, C.POINTER(Strategy), _P],
    "seemps_sweep": [_P, C.POINTER(ChainC), C.POINTER(SweepParams), C.POINTER(SweepReport)],
    "seemps_sweep_range": [_P, C.POINTER(ChainC), C.POINTER(SweepParams), _I, _I, _I,
                           C.POINTER(SweepReport)],
    "seemps_build_environments": [_P, C.POINTER(ChainC), _I, _I, _I],
    "seemps_sweep_batch": [C.POINTER(_P), C.POINTER(C.POINTER(ChainC)), C.POINTER(C.POINTER(SweepParams)),
                           _I, _I, C.POINTER(SweepReport), C.POINTER(_I)],
    "seemps_heff_apply_noalloc": [C.POINTER(PairDims), _P, _P, _P, _P, _P, _P, _P, C.c_char_p,
                                  C.c_size_t],
    "seemps_mlp_param_count": [_I, C.POINTER(_I)],
    "seemps_mlp_create": [C.POINTER(_P), _I, _P],
    "seemps_mlp_destroy": [_P],
    "seemps_mlp_set_site": [_P, _I, _I],
    "seemps_mlp_forward": [_P, _P, C.POINTER(PairDims), _P, _P, _P, _P, _P, _P],
    "seemps_mlp_loss_grad": [_P, _P, C.POINTER(PairDims), _P, _P, _P, _P, _P, _P, _P, _P],
    "seemps_mlp_adam": [_P, _P, _P, _P, _P, _I, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float],
    "seemps_mlp_train": [_P, _P, C.POINTER(MlpDataset), C.POINTER(MlpTrainParams), _P, _P, _P, C.POINTER(_I),
                         C.POINTER(C.c_double)],
    "seemps_svd_cleanup_stats": [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                 _I],
    "seemps_svd_stats": [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                         C.POINTER(C.c_double), _I],
    "seemps_svd_sweep_counts": [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), _I, C.POINTER(C.c_int)],
    "seemps_set_timing": [_P, _I],
    "seemps_autotune": [_P, C.POINTER(PairDims), C.POINTER(_I)],
    "seemps_set_autotune": [_P, _I],
    "seemps_autotune_stats": [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(_I)],
    "seemps_get_timing": [_P, C.POINTER(C.c_double), C.POINTER(C.c_longlong), _I],
}

PHASES = ["matvec", "tc_gemm", "local", "svd", "env", "jacobi", "qr"]
PHASE_COUNT = 8


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load the in-tree library (building it first if it is absent)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run the build first")
        _build.build()
    lib = C.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.seemps_last_error.argtypes = [_P]
    lib.seemps_last_error.restype = C.c_char_p
    _LIB = lib
    return lib


def _ptr(t) -> int:
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("tensor must live in CUDA device memory")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _f64(t):
    if t.dtype != torch.float64:
        raise ValueError("float64 tensor expected")
    return _ptr(t)


def workspace_bytes(chi_max: int, d: int, D_max: int, krylov_dim: int = 20, chib_max: int = 0) -> int:
    out = C.c_size_t(0)
    st = load().seemps_workspace_bytes(chi_max, d, D_max, krylov_dim, chib_max, C.byref(out))
    if st != OK:
        raise SeempsError(st, "workspace_bytes")
    return int(out.value)


@dataclass
class SvdResult:
    A_left: torch.Tensor    # (m, r)
    A_right: torch.Tensor   # (r, n)
    S: torch.Tensor         # (min(m, n),) descending
    rank: int
    discarded: float


class Context:
    """A library context bound to one device, one stream and one workspace."""

    def __init__(self, device: int = 0, chi_max: int = 64, d: int = 2, D_max: int = 5,
                 krylov_dim: int = 20, chib_max: int = 0, stream=None, workspace_bytes_=None):
        self.lib = load()
        self.device = torch.device("cuda", device)
        nbytes = workspace_bytes_ or workspace_bytes(chi_max, d, D_max, krylov_dim, chib_max)
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        st = self.lib.seemps_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream),
                                    C.c_void_p(self.workspace.data_ptr()), int(nbytes))
        if st != OK:
            raise SeempsError(st, "seemps_create")
        self.h = h
        self._scal = torch.zeros(8, dtype=torch.float64, device=self.device)
        self._iscal = torch.zeros(8, dtype=torch.int32, device=self.device)

    # -------------------------------------------------------------- plumbing
    def _check(self, st: int, what: str):
        if st != OK:
            msg = self.lib.seemps_last_error(self.h)
            raise SeempsError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.seemps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fused_mixing(self, enabled: bool):
        """MPO mixing of the bf16x3 effective operator in the first GEMM's epilogue, or in a kernel of
        its own (the default; seemps_set_fused_mixing); the results are bit-identical."""
        self._check(self.lib.seemps_set_fused_mixing(self.h, int(enabled)), "set_fused_mixing")

    def set_wait_limit(self, clocks: int):
        """Limit of the device-side software waits in SM clocks (seemps_set_wait_limit); -1 restores
        the default."""
        self._check(self.lib.seemps_set_wait_limit(self.h, int(clocks)), "set_wait_limit")

    def launch_count(self) -> int:
        c = C.c_longlong(0)
        self._check(self.lib.seemps_launch_count(self.h, C.byref(c)), "launch_count")
        return int(c.value)

    def device_status(self) -> int:
        s = C.c_int(0)
        self._check(self.lib.seemps_device_status(self.h, C.byref(s)), "device_status")
        return int(s.value)

    def _new(self, *shape):
        return torch.empty(*shape, dtype=torch.float64, device=self.device)

    # -------------------------------------------------------------- calls
    def env_update(self, side: int, E_in, A, W, precision: int = FP64, out=None):
        """Quadratic-form environment update (seemps_env_update)."""
        if side == LEFT:
            ci, d, co = A.shape
            Di, Do = W.shape[0], W.shape[3]
        else:
            co, d, ci = A.shape
            Do, Di = W.shape[0], W.shape[3]
        if out is None:  # double-FP64 environments: hi parts, then lo parts
            out = self._new(2, co, Do, co) if precision == FP64X2 else self._new(co, Do, co)
        self._check(self.lib.seemps_env_update(self.h, side, ci, co, d, Di, Do, _f64(E_in), _f64(A),
                                               _f64(W), _f64(out), precision), "env_update")
        return out

    def env_update_braket(self, side: int, E_in, X, B, W, precision: int = FP64, out=None):
        """Environment of <x, W b> (seemps_env_update_braket); X is x's tensor, B is b's."""
        if side == LEFT:
            cix, d, cox = X.shape
            cib, _, cob = B.shape
            Di, Do = W.shape[0], W.shape[3]
        else:
            cox, d, cix = X.shape
            cob, _, cib = B.shape
            Do, Di = W.shape[0], W.shape[3]
        out = out if out is not None else self._new(cox, Do, cob)
        self._check(self.lib.seemps_env_update_braket(self.h, side, cix, cib, cox, cob, d, Di, Do, _f64(E_in),
                                                      _f64(X), _f64(B), _f64(W), _f64(out), precision),
                    "env_update_braket")
        return out

    def env_update_linear(self, side: int, F_in, A, B, out=None):
        """Antilinear-form environment update (seemps_env_update_linear)."""
        if side == LEFT:
            ci, d, co = A.shape
            bi, _, bo = B.shape
        else:
            co, d, ci = A.shape
            bo, _, bi = B.shape
        out = out if out is not None else self._new(co, bo)
        self._check(self.lib.seemps_env_update_linear(self.h, side, ci, co, bi, bo, d, _f64(F_in),
                                                      _f64(A), _f64(B), _f64(out)), "env_update_linear")
        return out

    def two_site(self, A1, A2, out=None):
        chl, d, chm = A1.shape
        chr_ = A2.shape[2]
        out = out if out is not None else self._new(chl, d, d, chr_)
        self._check(self.lib.seemps_two_site(self.h, chl, chm, chr_, d, _f64(A1), _f64(A2), _f64(out)),
                    "two_site")
        return out

    @staticmethod
    def _dims(L, W1, W2, R):
        # L, R are (chi, D, chi), or (2, chi, D, chi) in double-FP64 (hi parts, lo parts)
        return PairDims(L.shape[-3], R.shape[-3], W1.shape[1], W1.shape[0], W1.shape[3], W2.shape[3])

    def heff_apply(self, L, W1, W2, R, theta, precision: int = FP64, out=None):
        dm = self._dims(L, W1, W2, R)
        out = out if out is not None else torch.empty_like(theta)
        self._check(self.lib.seemps_heff_apply(self.h, C.byref(dm), _f64(L), _f64(W1), _f64(W2), _f64(R),
                                               _f64(theta), _f64(out), precision), "heff_apply")
        return out

    def heff1_apply(self, L, W, R, A, precision: int = FP64, out=None):
        """One-site effective operator H^(site) A (seemps_heff1_apply); A is (chi_l, d, chi_r)."""
        dm = PairDims(L.shape[0], R.shape[0], W.shape[1], W.shape[0], W.shape[3], W.shape[3])
        out = out if out is not None else torch.empty_like(A)
        self._check(self.lib.seemps_heff1_apply(self.h, C.byref(dm), _f64(L), _f64(W), _f64(R), _f64(A),
                                                _f64(out), precision), "heff1_apply")
        return out

    def local_expm(self, L, W1, W2, R, theta, tau: float, krylov_dim: int = 20, breakdown_tol: float = 1e-14,
                   precision: int = FP64):
        """theta <- exp(tau H) theta / |.| in place (seemps_local_expm); W2 None for the one-site
        operator.  Returns (<theta, H theta>/<theta, theta> of the input, Krylov steps)."""
        if W2 is None:
            dm = PairDims(L.shape[0], R.shape[0], W1.shape[1], W1.shape[0], W1.shape[3], W1.shape[3])
            sites, w2 = 1, None
        else:
            dm = self._dims(L, W1, W2, R)
            sites, w2 = 2, _f64(W2)
        e, it = self._scal[0:1], self._iscal[0:1]
        self._check(self.lib.seemps_local_expm(self.h, C.byref(dm), sites, _f64(L), _f64(W1), w2, _f64(R),
                                               _f64(theta), krylov_dim, breakdown_tol, tau, precision,
                                               _ptr(e), _ptr(it)), "local_expm")
        return float(e.item()), int(it.item())

    def heff_apply_braket(self, L, W1, W2, R, theta_b, precision: int = FP64, out=None):
        """The pair's MPO action between x's bonds (L, R first index) and b's (theta_b):
        seemps_heff_apply_braket; returns y (chi_l, d, d, chi_r)."""
        dm = self._dims(L, W1, W2, R)
        out = out if out is not None else self._new(dm.chi_l, dm.d, dm.d, dm.chi_r)
        self._check(self.lib.seemps_heff_apply_braket(self.h, C.byref(dm), theta_b.shape[0], theta_b.shape[3],
                                                      _f64(L), _f64(W1), _f64(W2), _f64(R), _f64(theta_b),
                                                      _f64(out), precision), "heff_apply_braket")
        return out

    def heff_diagonal(self, L, W1, W2, R, out=None):
        dm = self._dims(L, W1, W2, R)
        out = out if out is not None else self._new(dm.chi_l, dm.d, dm.d, dm.chi_r)
        self._check(self.lib.seemps_heff_diagonal(self.h, C.byref(dm), _f64(L), _f64(W1), _f64(W2),
                                                  _f64(R), _f64(out)), "heff_diagonal")
        return out

    def b_effective(self, F, B1, B2, G, out=None):
        chl, chr_ = F.shape[0], G.shape[0]
        bl, d, bm = B1.shape
        br = B2.shape[2]
        out = out if out is not None else self._new(chl, d, d, chr_)
        self._check(self.lib.seemps_b_effective(self.h, chl, chr_, bl, bm, br, d, _f64(F), _f64(B1),
                                                _f64(B2), _f64(G), _f64(out)), "b_effective")
        return out

    def local_eig(self, L, W1, W2, R, theta, krylov_dim: int = 20, breakdown_tol: float = 1e-14,
                  precision: int = FP64):
        """Lanczos on H_n from theta (in place); returns (energy, steps) read back to the host."""
        dm = self._dims(L, W1, W2, R)
        e, it = self._scal[0:1], self._iscal[0:1]
        self._check(self.lib.seemps_local_eig(self.h, C.byref(dm), _f64(L), _f64(W1), _f64(W2), _f64(R),
                                              _f64(theta), krylov_dim, breakdown_tol, precision,
                                              _ptr(e), _ptr(it)), "local_eig")
        return float(e.item()), int(it.item())

    def local_pcg(self, L, W1, W2, R, b, x, precond: int = PRECOND_JACOBI, rtol: float = 1e-12,
                  maxiter: int = 500, precision: int = FP64, mlp=None, site=None, n_sites=None):
        """PCG on H_n x = b from x (in place); returns (relative residual, iterations)."""
        dm = self._dims(L, W1, W2, R)
        res, it = self._scal[1:2], self._iscal[1:2]
        mptr = mlp.handle if mlp is not None else None
        if mlp is not None and site is not None:
            mlp.set_site(site, n_sites)
        self._check(self.lib.seemps_local_pcg(self.h, C.byref(dm), _f64(L), _f64(W1), _f64(W2), _f64(R),
                                              _f64(b), _f64(x), precond, mptr, rtol, maxiter, precision,
                                              _ptr(res), _ptr(it)), "local_pcg")
        return float(res.item()), int(it.item())

    def cgs_solve(self, W: list, B: list, X0: list, chi_max: int, tol: float = 1e-14, rule: int = TRUNC_WEIGHT,
                  rtol: float = 1e-10, maxiter: int = 100, n_sweeps: int = 2, precision: int = FP64):
        """Conjugate gradients on MPS for U x = b (seemps_cgs_solve).  W, B, X0: lists of
        site tensors (numpy or torch).  Returns (x tensors, report dict)."""
        dev = self.device
        N, d = len(B), int(B[0].shape[1])
        Wt = [torch.as_tensor(w, dtype=torch.float64).to(dev).contiguous() for w in W]
        Bt = [torch.as_tensor(b, dtype=torch.float64).to(dev).contiguous() for b in B]
        Dl = [1] + [int(w.shape[3]) for w in W]
        chib = [1] + [int(b.shape[2]) for b in B]
        chix = [1] + [int(x.shape[2]) for x in X0]
        cx = max(chi_max, max(chix))  # a larger guess bond is refused by the library, not here
        cap = cx * d * cx
        Xb = []
        for x in X0:
            buf = torch.zeros(cap, dtype=torch.float64, device=dev)
            t = torch.as_tensor(x, dtype=torch.float64).reshape(-1)
            buf[: t.numel()] = t.to(dev)
            Xb.append(buf)
        nbytes = C.c_size_t(0)
        st = self.lib.seemps_cgs_work_bytes(N, d, max(Dl), chi_max, max(chib), C.byref(nbytes))
        if st != OK:
            raise SeempsError(st, "cgs_work_bytes")
        work = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)

        def parr(ts):
            return (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

        Da, cba, cxa = (C.c_int * (N + 1))(*Dl), (C.c_int * (N + 1))(*chib), (C.c_int * (N + 1))(*chix)
        Wa, Ba, Xa = parr(Wt), parr(Bt), parr(Xb)
        pr = CgsProblem(N, d, C.cast(Da, C.POINTER(C.c_int)), C.cast(Wa, C.POINTER(C.c_void_p)),
                        C.cast(cba, C.POINTER(C.c_int)), C.cast(Ba, C.POINTER(C.c_void_p)),
                        C.cast(cxa, C.POINTER(C.c_int)), C.cast(Xa, C.POINTER(C.c_void_p)),
                        C.c_void_p(work.data_ptr()), nbytes.value)
        prm = CgsParams(Strategy(chi_max, tol, rule), n_sweeps, precision, maxiter, rtol)
        hist = (C.c_double * (maxiter + 1))()
        rep = CgsReport(0, 0.0, 0.0, 0.0, C.cast(hist, C.POINTER(C.c_double)))
        self._check(self.lib.seemps_cgs_solve(self.h, C.byref(pr), C.byref(prm), C.byref(rep)), "cgs_solve")
        chis = [int(cxa[i]) for i in range(N + 1)]
        x = [Xb[i][: chis[i] * d * chis[i + 1]].view(chis[i], d, chis[i + 1]) for i in range(N)]
        return x, {"iterations": rep.iterations, "residual": rep.residual, "norm_b": rep.norm_b,
                   "seconds": rep.seconds, "residual_history": list(hist[: rep.iterations + 1])}

    def autotune(self, chi_l: int, chi_r: int, d: int, D_l: int, D_m: int, D_r: int) -> int:
        """Time both tile shapes on the bf16x3 GEMMs of a pair update at these sizes (seemps_autotune);
        returns the number of shapes newly timed."""
        n = C.c_int(0)
        dm = PairDims(chi_l, chi_r, d, D_l, D_m, D_r)
        self._check(self.lib.seemps_autotune(self.h, C.byref(dm), C.byref(n)), "autotune")
        return int(n.value)

    def set_autotune(self, enabled: bool):
        self._check(self.lib.seemps_set_autotune(self.h, int(enabled)), "set_autotune")

    def autotune_stats(self) -> dict:
        hits, shapes, size = C.c_longlong(0), C.c_longlong(0), C.c_int(0)
        self._check(self.lib.seemps_autotune_stats(self.h, C.byref(hits), C.byref(shapes), C.byref(size)),
                    "autotune_stats")
        return {"hits": int(hits.value), "shapes_timed": int(shapes.value), "table_size": int(size.value)}

    def set_timing(self, enabled: bool):
        self._check(self.lib.seemps_set_timing(self.h, int(enabled)), "set_timing")

    def svd_stats(self, reset: bool = False) -> dict:
        calls, sweeps, pairs = C.c_longlong(0), C.c_longlong(0), C.c_longlong(0)
        flops = C.c_double(0.0)
        self._check(self.lib.seemps_svd_stats(self.h, C.byref(calls), C.byref(sweeps), C.byref(pairs),
                                              C.byref(flops), int(reset)), "svd_stats")
        return {"calls": calls.value, "sweeps": sweeps.value, "pair_visits": pairs.value, "flops": flops.value}

    def svd_cleanup_stats(self, reset: bool = False) -> dict:
        """Splits that finished with the Jacobi cleanup phase, its rounds and fallbacks."""
        calls, rounds, fb = C.c_longlong(0), C.c_longlong(0), C.c_longlong(0)
        self._check(self.lib.seemps_svd_cleanup_stats(self.h, C.byref(calls), C.byref(rounds), C.byref(fb),
                                                      int(reset)), "svd_cleanup_stats")
        return {"calls": calls.value, "rounds": rounds.value, "fallbacks": fb.value}

    def svd_sweep_counts(self) -> tuple:
        """(rotations, visits) per sweep of the most recent large-problem Jacobi SVD."""
        cap = 256
        rot, vis, n = (C.c_int * cap)(), (C.c_int * cap)(), C.c_int(0)
        self._check(self.lib.seemps_svd_sweep_counts(self.h, rot, vis, cap, C.byref(n)), "svd_sweep_counts")
        k = min(n.value, cap)
        return list(rot[:k]), list(vis[:k])

    def get_timing(self, reset: bool = False) -> dict:
        """{phase: (total ms, intervals)} from the per-phase CUDA events."""
        ms = (C.c_double * PHASE_COUNT)()
        cnt = (C.c_longlong * PHASE_COUNT)()
        self._check(self.lib.seemps_get_timing(self.h, ms, cnt, int(reset)), "get_timing")
        return {name: (ms[i], int(cnt[i])) for i, name in enumerate(PHASES)}

    def svd_truncate(self, M, chi_max: int, tol: float, rule: int = TRUNC_WEIGHT,
                     absorb: int = ABSORB_RIGHT, normalize: bool = False, max_sweeps: int = 0,
                     precision: int = FP64) -> SvdResult:
        m, n = M.shape
        p = min(m, n)
        rmax = min(p, chi_max)
        Al = self._new(m * rmax)
        Ar = self._new(rmax * n)
        S = self._new(p)
        st = Strategy(chi_max, tol, rule)
        rank, disc = self._iscal[2:3], self._scal[2:3]
        self._check(self.lib.seemps_svd_truncate(self.h, m, n, _f64(M), C.byref(st), absorb, int(normalize),
                                                 _f64(Al), _f64(Ar), _f64(S), _ptr(rank), _ptr(disc),
                                                 max_sweeps, precision), "svd_truncate")
        r = int(rank.item())
        return SvdResult(Al[: m * r].view(m, r), Ar[: r * n].view(r, n), S, r, float(disc.item()))

    def truncation_rank(self, s, chi_max: int, tol: float, rule: int = TRUNC_WEIGHT) -> int:
        st = Strategy(chi_max, tol, rule)
        rank = self._iscal[3:4]
        self._check(self.lib.seemps_truncation_rank(self.h, s.numel(), _f64(s), C.byref(st), _ptr(rank)),
                    "truncation_rank")
        return int(rank.item())

    @staticmethod
    def _params(mode, n_sweeps, refine_sweeps, precision, krylov_dim, breakdown_tol, chi_max, tol, rule,
                canonicalize, pcg_rtol, pcg_maxiter, precond, mlp, tdvp_dt=0.0):
        return SweepParams(mode, n_sweeps, refine_sweeps, precision, krylov_dim, breakdown_tol,
                           Strategy(chi_max, tol, rule), int(canonicalize), pcg_rtol, pcg_maxiter, precond,
                           mlp.handle if mlp is not None else None, tdvp_dt)

    def build_environments(self, chain: "Chain", first: int, mode: int = MODE_EIG, precision: int = FP64):
        cc = chain.c_struct()
        self._check(self.lib.seemps_build_environments(self.h, C.byref(cc), mode, first, precision),
                    "build_environments")

    def sweep_range(self, chain: "Chain", first: int, count: int, direction: int = 1, mode: int = MODE_EIG,
                    precision: int = FP64, krylov_dim: int = 20, breakdown_tol: float = 1e-14,
                    chi_max: int = 64, tol: float = 1e-12, rule: int = TRUNC_WEIGHT, pcg_rtol: float = 1e-12,
                    pcg_maxiter: int = 500, precond: int = PRECOND_JACOBI, mlp=None, tdvp_dt: float = 0.0):
        """`count` pair updates from pair `first` (seemps_sweep_range); returns a dict report."""
        p = self._params(mode, 0, 0, precision, krylov_dim, breakdown_tol, chi_max, tol, rule, False,
                         pcg_rtol, pcg_maxiter, precond, mlp, tdvp_dt)
        rep = SweepReport(0.0, 0.0, 0.0, 0, 0.0, 0, None, None)
        cc = chain.c_struct()
        self._check(self.lib.seemps_sweep_range(self.h, C.byref(cc), C.byref(p), first, count, direction,
                                                C.byref(rep)), "sweep_range")
        chain.pull_dims(cc)
        return {"energy": rep.energy, "max_discarded": rep.max_discarded, "error_bound": rep.error_bound,
                "local_iters": int(rep.local_iters), "seconds": rep.seconds}

    def sweep(self, chain: "Chain", mode: int = MODE_EIG, n_sweeps: int = 1, refine_sweeps: int = 0,
              precision: int = FP64, krylov_dim: int = 20, breakdown_tol: float = 1e-14,
              chi_max: int = 64, tol: float = 1e-12, rule: int = TRUNC_WEIGHT, canonicalize: bool = True,
              pcg_rtol: float = 1e-12, pcg_maxiter: int = 500, precond: int = PRECOND_JACOBI, mlp=None,
              tdvp_dt: float = 0.0):
        """Full sweeps over a Chain (seemps_sweep); returns a dict report.  In TDVP mode each sweep
        is one time step tdvp_dt of imaginary time."""
        p = self._params(mode, n_sweeps, refine_sweeps, precision, krylov_dim, breakdown_tol, chi_max, tol,
                         rule, canonicalize, pcg_rtol, pcg_maxiter, precond, mlp, tdvp_dt)
        nh = 2 * (n_sweeps + refine_sweeps)
        he = (C.c_double * max(1, nh))()
        hr = (C.c_int * max(1, nh))()
        rep = SweepReport(0.0, 0.0, 0.0, 0, 0.0, 0, C.cast(he, C.POINTER(C.c_double)),
                          C.cast(hr, C.POINTER(C.c_int)))
        cc = chain.c_struct()
        self._check(self.lib.seemps_sweep(self.h, C.byref(cc), C.byref(p), C.byref(rep)), "sweep")
        chain.pull_dims(cc)
        return {"energy": rep.energy, "max_discarded": rep.max_discarded, "error_bound": rep.error_bound,
                "local_iters": int(rep.local_iters), "seconds": rep.seconds, "half_sweeps": rep.half_sweeps,
                "half_sweep_energy": list(he)[:nh], "half_sweep_max_rank": list(hr)[:nh]}


class Chain:
    """Device buffers of one chain for seemps_sweep (MPS, MPO, environments)."""

    def __init__(self, ctx: Context, W: list, A: list, chi_max: int, B: list = None, extended: bool = False):
        """W = None builds a chain without MPO and quadratic environments (simplify mode);
        extended = True sizes the quadratic environments for FP64X2 sweeps (double-FP64)."""
        dev = ctx.device
        self.N = len(A)
        self.d = A[0].shape[1]
        self.chi_max = chi_max
        self.Dlist = None if W is None else [1] + [int(w.shape[3]) for w in W]
        self.W = None if W is None else [torch.as_tensor(w, dtype=torch.float64).to(dev).contiguous() for w in W]
        chi = [1] + [int(a.shape[2]) for a in A]
        cap_chi = max(chi_max, max(chi))
        self.chi = chi
        self.A = []
        for a in A:
            buf = torch.zeros(cap_chi * self.d * cap_chi, dtype=torch.float64, device=dev)
            t = torch.as_tensor(a, dtype=torch.float64).reshape(-1)
            buf[: t.numel()] = t.to(dev)
            self.A.append(buf)
        self.L = self.R = None
        bmax = 1 if B is None else max([1] + [int(b.shape[2]) for b in B])
        if W is not None:
            # room for (chi, D, chi) and, in apply mode, (chi, D, chib) environments
            envn = cap_chi * max(self.Dlist) * max(cap_chi, bmax) * (2 if extended else 1)
            self.L = [torch.zeros(envn, dtype=torch.float64, device=dev) for _ in range(self.N + 1)]
            self.R = [torch.zeros(envn, dtype=torch.float64, device=dev) for _ in range(self.N + 1)]
        self.B = None
        if B is not None:
            self.B = [torch.as_tensor(b, dtype=torch.float64).to(dev).contiguous() for b in B]
            self.chib = [1] + [int(b.shape[2]) for b in B]
            bmax = max(self.chib)
            self.F = [torch.zeros(cap_chi * bmax, dtype=torch.float64, device=dev) for _ in range(self.N + 1)]
            self.G = [torch.zeros(cap_chi * bmax, dtype=torch.float64, device=dev) for _ in range(self.N + 1)]

    def c_struct(self) -> ChainC:
        def parr(ts):
            return (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

        self._keep = []
        chi = (C.c_int * (self.N + 1))(*self.chi)
        A = parr(self.A)
        self._keep += [chi, A]
        cc = ChainC(self.N, self.d, None, None, C.cast(A, C.POINTER(C.c_void_p)), C.cast(chi, C.POINTER(C.c_int)),
                    None, None, None, None, None, None)
        if self.W is not None:
            D = (C.c_int * (self.N + 1))(*self.Dlist)
            W, L, R = parr(self.W), parr(self.L), parr(self.R)
            self._keep += [D, W, L, R]
            cc.D = C.cast(D, C.POINTER(C.c_int))
            cc.W = C.cast(W, C.POINTER(C.c_void_p))
            cc.Lenv = C.cast(L, C.POINTER(C.c_void_p))
            cc.Renv = C.cast(R, C.POINTER(C.c_void_p))
        if self.B is not None:
            B, F, G = parr(self.B), parr(self.F), parr(self.G)
            chib = (C.c_int * (self.N + 1))(*self.chib)
            self._keep += [B, F, G, chib]
            cc.B = C.cast(B, C.POINTER(C.c_void_p))
            cc.chib = C.cast(chib, C.POINTER(C.c_int))
            cc.Fenv = C.cast(F, C.POINTER(C.c_void_p))
            cc.Genv = C.cast(G, C.POINTER(C.c_void_p))
        self._chi_arr = chi
        return cc

    def pull_dims(self, cc: ChainC):
        self.chi = [int(self._chi_arr[i]) for i in range(self.N + 1)]

    def tensors(self) -> list:
        """Current MPS tensors as (chi_l, d, chi_r) views."""
        out = []
        for i in range(self.N):
            n = self.chi[i] * self.d * self.chi[i + 1]
            out.append(self.A[i][:n].view(self.chi[i], self.d, self.chi[i + 1]))
        return out


class Mlp:
    """The learned preconditioner: float32 parameters on the device plus the
    Adam moments and a gradient accumulator (seemps_mlp_*)."""

    HIDDEN = 64

    def __init__(self, ctx: Context, params):
        self.ctx = ctx
        self.lib = ctx.lib
        n = C.c_int(0)
        st = self.lib.seemps_mlp_param_count(self.HIDDEN, C.byref(n))
        if st != OK:
            raise SeempsError(st, "mlp_param_count")
        self.n = n.value
        self.params = torch.as_tensor(params, dtype=torch.float32).to(ctx.device).contiguous()
        if self.params.numel() != self.n:
            raise ValueError(f"expected {self.n} parameters")
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float64, device=ctx.device)
        self.t = 0
        h = C.c_void_p()
        st = self.lib.seemps_mlp_create(C.byref(h), self.HIDDEN, C.c_void_p(self.params.data_ptr()))
        if st != OK:
            raise SeempsError(st, "mlp_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.seemps_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_site(self, site: int, n_sites: int):
        self.ctx._check(self.lib.seemps_mlp_set_site(self.handle, site, n_sites), "mlp_set_site")

    def forward(self, L, W1, W2, R):
        dm = Context._dims(L, W1, W2, R)
        n = dm.chi_l * dm.d * dm.d * dm.chi_r
        p = torch.empty(n, dtype=torch.float64, device=self.ctx.device)
        U = torch.empty(n, 4, dtype=torch.float64, device=self.ctx.device)
        self.ctx._check(self.lib.seemps_mlp_forward(self.ctx.h, self.handle, C.byref(dm), _f64(L), _f64(W1),
                                                    _f64(W2), _f64(R), _f64(p), _f64(U)), "mlp_forward")
        return p, U

    def zero_grad(self):
        self.grad.zero_()
        self.loss.zero_()

    def loss_grad(self, L, W1, W2, R, b, xstar):
        """Adds this system's loss and gradient to the accumulators."""
        dm = Context._dims(L, W1, W2, R)
        self.ctx._check(self.lib.seemps_mlp_loss_grad(self.ctx.h, self.handle, C.byref(dm), _f64(L), _f64(W1),
                                                      _f64(W2), _f64(R), _f64(b), _f64(xstar),
                                                      _ptr(self.grad), _ptr(self.loss)), "mlp_loss_grad")

    def train(self, systems: list, steps: int, lr: float = 3e-3, batch: int = 0, beta1=0.9, beta2=0.999,
              eps=1e-8, history: bool = False) -> list:
        """seemps_mlp_train on systems (objects with L, W1, W2, R, b, xstar device tensors and
        site, n_sites); returns the per-step mean losses when history is set."""
        n = len(systems)
        ptr = lambda ts: (C.c_void_p * n)(*[_f64(t) for t in ts])  # noqa: E731
        dims = (PairDims * n)(*[Context._dims(s.L, s.W1, s.W2, s.R) for s in systems])
        arrs = [ptr([getattr(s, f) for s in systems]) for f in ("L", "W1", "W2", "R", "b", "xstar")]
        site = (C.c_int * n)(*[s.site for s in systems])
        nsit = (C.c_int * n)(*[s.n_sites for s in systems])
        ds = MlpDataset(n, C.cast(dims, C.POINTER(PairDims)), *[C.cast(a, C.POINTER(C.c_void_p)) for a in arrs],
                        C.cast(site, C.POINTER(C.c_int)), C.cast(nsit, C.POINTER(C.c_int)))
        tp = MlpTrainParams(steps, batch, lr, beta1, beta2, eps)
        t = C.c_int(self.t)
        hist = (C.c_double * max(1, steps))() if history else None
        self.ctx._check(self.lib.seemps_mlp_train(self.ctx.h, self.handle, C.byref(ds), C.byref(tp), _ptr(self.grad),
                                                  _ptr(self.m), _ptr(self.v), C.byref(t), hist), "mlp_train")
        self.t = t.value
        return list(hist)[:steps] if history else []

    def adam_step(self, lr: float, grad_scale: float = 1.0, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        self.ctx._check(self.lib.seemps_mlp_adam(self.ctx.h, self.handle, _ptr(self.grad), _ptr(self.m),
                                                 _ptr(self.v), self.t, lr, beta1, beta2, eps, grad_scale),
                        "mlp_adam")


def sweep_batch(ctxs: list, chains: list, params: list, max_threads: int = 0) -> list:
    """seemps_sweep_batch: chain k on ctxs[k] with params[k] (dicts of Context.sweep keywords).

    Returns one report dict per chain."""
    lib = load()
    n = len(chains)
    assert len(ctxs) == n and len(params) == n
    ps = [Context._params(kw.get("mode", MODE_EIG), kw.get("n_sweeps", 1), kw.get("refine_sweeps", 0),
                          kw.get("precision", FP64), kw.get("krylov_dim", 20), kw.get("breakdown_tol", 1e-14),
                          kw.get("chi_max", 64), kw.get("tol", 1e-12), kw.get("rule", TRUNC_WEIGHT),
                          kw.get("canonicalize", True), kw.get("pcg_rtol", 1e-12), kw.get("pcg_maxiter", 500),
                          kw.get("precond", PRECOND_JACOBI), kw.get("mlp"), kw.get("tdvp_dt", 0.0))
          for kw in params]
    ccs = [ch.c_struct() for ch in chains]
    cptr = (C.c_void_p * n)(*[c.h.value for c in ctxs])
    chptr = (C.POINTER(ChainC) * n)(*[C.pointer(cc) for cc in ccs])
    pptr = (C.POINTER(SweepParams) * n)(*[C.pointer(p) for p in ps])
    hes = [(C.c_double * max(1, 2 * (kw.get("n_sweeps", 1) + kw.get("refine_sweeps", 0))))() for kw in params]
    reps = (SweepReport * n)()
    for k in range(n):
        reps[k].half_sweep_energy = C.cast(hes[k], C.POINTER(C.c_double))
    sts = (C.c_int * n)()
    st = lib.seemps_sweep_batch(cptr, chptr, pptr, n, max_threads, reps, sts)
    for k in range(n):
        chains[k].pull_dims(ccs[k])
    if st != OK:
        bad = [k for k in range(n) if sts[k] != OK]
        if not bad:  # refused before any chain ran (e.g. a context shared by two chains)
            raise SeempsError(st, "sweep_batch: invalid arguments")
        raise SeempsError(st, f"sweep_batch: chain {bad[0]}: {lib.seemps_last_error(ctxs[bad[0]].h).decode()}")
    return [{"energy": reps[k].energy, "max_discarded": reps[k].max_discarded, "error_bound": reps[k].error_bound,
             "local_iters": int(reps[k].local_iters), "seconds": reps[k].seconds,
             "half_sweep_energy": list(hes[k])} for k in range(n)]
