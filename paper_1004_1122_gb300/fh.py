"""ctypes binding of libfh.so (C ABI in include/fh.h).

Argument marshalling only: every step of the operator and the solvers runs in
the CUDA library.  PyTorch provides device memory and the CUDA stream.  If the
library is missing the import of a Solver fails loudly; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libfh.so")
# Launch-shape cache read by fh_create and written by fh_autotune (see fh.h).
# The package ships the shapes tuned on GB300 for its benchmark grids as a
# read-only seed; runs read and append to a private copy next to the built
# library (never to the shipped file), unless FH_TUNE_CACHE names another file.
TUNE_SEED = os.path.join(_HERE, "tune_cache.txt")
TUNE_CACHE = os.path.join(_HERE, "lib", "tune_cache.txt")


def _default_tune_cache() -> str:
    if not os.path.exists(TUNE_CACHE):
        try:
            os.makedirs(os.path.dirname(TUNE_CACHE), exist_ok=True)
            with open(TUNE_SEED) as src, open(TUNE_CACHE, "x") as dst:
                dst.write(src.read())
        except FileExistsError:
            pass
        except OSError:  # read-only install: read the seed, tune results are not kept
            return TUNE_SEED
    return TUNE_CACHE


if "FH_TUNE_CACHE" not in os.environ:
    os.environ["FH_TUNE_CACHE"] = _default_tune_cache()

FH_OK = 0
STATUS = {
    0: "FH_OK", 1: "FH_ERR_ARG", 2: "FH_ERR_EVEN_N", 3: "FH_ERR_NOT_SPD", 4: "FH_ERR_OOM",
    5: "FH_ERR_CUDA", 6: "FH_ERR_NOT_CONVERGED", 7: "FH_ERR_BREAKDOWN", 8: "FH_ERR_TIMEOUT",
    9: "FH_ERR_UNSUPPORTED",
}
METHODS = {"cg": 0, "bicg": 1, "fixed_point": 2, "ffth": 2}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_refined": 2}
DT_FP64, DT_FP32 = 0, 1

# Names declared in include/fh.h (checked by the ABI test).
EXPORTS = (
    "fh_create", "fh_set_phase", "fh_apply", "fh_solve", "fh_solve_all", "fh_effective_column",
    "fh_eta_e", "fh_profile", "fh_autotune", "fh_apply_noalloc", "fh_batch_create", "fh_batch_solve",
    "fh_batch_last_error", "fh_batch_destroy", "fh_project_compatible", "fh_autotune_loads",
    "fh_batch_autotune", "fh_destroy", "fh_status_string", "fh_last_error",
    "fh_version", "fh_set_wait_limit", "fh_wait_selftest",
    # fh_nn.h
    "fh_nn_create", "fh_nn_param_count", "fh_nn_launches", "fh_nn_set_params", "fh_nn_get_params",
    "fh_nn_forward", "fh_nn_gradients", "fh_nn_train_step", "fh_nn_destroy", "fh_nn_features",
    "fh_nn_targets", "fh_nn_warm_start", "fh_nn_response_features",
)


class FhInfo(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("outer_iters", ctypes.c_int),
        ("matvecs", ctypes.c_int),
        ("status", ctypes.c_int),
        ("rel_res_true", ctypes.c_double),
        ("rel_res", ctypes.c_double),
        ("eta_r", ctypes.c_double),
        ("eta_e", ctypes.c_double),
        ("history", ctypes.POINTER(ctypes.c_double)),
        ("history_cap", ctypes.c_int),
        ("history_len", ctypes.c_int),
        ("launches", ctypes.c_longlong),
        ("flags", ctypes.c_int),
        ("ct_plans", ctypes.c_int),
        ("eta_e_history", ctypes.POINTER(ctypes.c_double)),
        ("eta_r_history", ctypes.POINTER(ctypes.c_double)),
        ("eta_e_len", ctypes.c_int),
        ("eta_r_len", ctypes.c_int),
    ]


CT_PLANS = {1: 2187, 2: 729, 4: 243}  # fh_info.ct_plans bits (FH_CT_*)


class FhError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libfh.so and declare the prototypes.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(
            f"{path} not found: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    pI = ctypes.POINTER(ctypes.c_int)
    pD = ctypes.POINTER(ctypes.c_double)
    lib.fh_create.argtypes = [ctypes.POINTER(P), I, pI, pD, P, I, I, pD, pD, I, P]
    lib.fh_create.restype = I
    lib.fh_set_phase.argtypes = [P, P, I]
    lib.fh_set_phase.restype = I
    lib.fh_apply.argtypes = [P, P, P, I, I]
    lib.fh_apply.restype = I
    lib.fh_solve.argtypes = [P, pD, D, I, I, P, P, pD, ctypes.POINTER(FhInfo)]
    lib.fh_solve.restype = I
    lib.fh_solve_all.argtypes = [P, D, I, I, pD, ctypes.POINTER(FhInfo)]
    lib.fh_solve_all.restype = I
    lib.fh_effective_column.argtypes = [P, P, pD]
    lib.fh_effective_column.restype = I
    lib.fh_eta_e.argtypes = [P, P, pD]
    lib.fh_eta_e.restype = I
    lib.fh_profile.argtypes = [P, I, I, I, pD]
    lib.fh_profile.restype = I
    lib.fh_batch_create.argtypes = [ctypes.POINTER(P), I, pI, ctypes.POINTER(ctypes.c_void_p), pI,
                                    ctypes.POINTER(ctypes.c_void_p), I, I]
    lib.fh_batch_create.restype = I
    lib.fh_batch_solve.argtypes = [P, pD, D, I, I, pD, pI, pI, ctypes.POINTER(FhInfo)]
    lib.fh_batch_solve.restype = I
    lib.fh_batch_last_error.argtypes = [P]
    lib.fh_batch_last_error.restype = ctypes.c_char_p
    lib.fh_batch_destroy.argtypes = [P]
    lib.fh_batch_destroy.restype = V
    lib.fh_project_compatible.argtypes = [P, P, P]
    lib.fh_project_compatible.restype = I
    LL = ctypes.c_longlong
    pF = ctypes.POINTER(ctypes.c_float)
    lib.fh_nn_create.argtypes = [ctypes.POINTER(P), pI, I, I, pI, P]
    lib.fh_nn_create.restype = I
    lib.fh_nn_param_count.argtypes = [P]
    lib.fh_nn_param_count.restype = LL
    lib.fh_nn_launches.argtypes = [P]
    lib.fh_nn_launches.restype = LL
    lib.fh_nn_set_params.argtypes = [P, pF, LL]
    lib.fh_nn_set_params.restype = I
    lib.fh_nn_get_params.argtypes = [P, pF, LL]
    lib.fh_nn_get_params.restype = I
    lib.fh_nn_forward.argtypes = [P, P, P]
    lib.fh_nn_forward.restype = I
    lib.fh_nn_gradients.argtypes = [P, P, P, pD, pF]
    lib.fh_nn_gradients.restype = I
    lib.fh_nn_train_step.argtypes = [P, P, P, ctypes.c_float, I, pD]
    lib.fh_nn_train_step.restype = I
    lib.fh_nn_destroy.argtypes = [P]
    lib.fh_nn_destroy.restype = V
    lib.fh_nn_features.argtypes = [P, I, pD, I, LL, P, P]
    lib.fh_nn_features.restype = I
    lib.fh_nn_targets.argtypes = [ctypes.POINTER(ctypes.c_void_p), I, LL, P, P, P]
    lib.fh_nn_targets.restype = I
    lib.fh_nn_response_features.argtypes = [P, I, LL, P]
    lib.fh_nn_response_features.restype = I
    lib.fh_nn_warm_start.argtypes = [P, P, P, pD, I, LL, P, P]
    lib.fh_nn_warm_start.restype = I
    lib.fh_batch_autotune.argtypes = [P, pD, pD]
    lib.fh_batch_autotune.restype = I
    lib.fh_autotune_loads.argtypes = [P, pD, pD]
    lib.fh_autotune_loads.restype = I
    lib.fh_autotune.argtypes = [P, I, pD, pD]
    lib.fh_autotune.restype = I
    lib.fh_apply_noalloc.argtypes = [I, pI, pD, P, I, pD, pD, P, P, I, P, ctypes.c_char_p, ctypes.c_size_t]
    lib.fh_apply_noalloc.restype = I
    lib.fh_destroy.argtypes = [P]
    lib.fh_destroy.restype = V
    lib.fh_status_string.argtypes = [I]
    lib.fh_status_string.restype = ctypes.c_char_p
    lib.fh_last_error.argtypes = [P]
    lib.fh_last_error.restype = ctypes.c_char_p
    lib.fh_version.argtypes = []
    lib.fh_version.restype = ctypes.c_char_p
    lib.fh_set_wait_limit.argtypes = [D]
    lib.fh_set_wait_limit.restype = I
    lib.fh_wait_selftest.argtypes = [D, P]
    lib.fh_wait_selftest.restype = I
    _lib = lib
    return lib


def _dptr(a) -> ctypes.c_double:
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _info_dict(info: FhInfo, hist: Optional[np.ndarray], eta_e_h: Optional[np.ndarray] = None,
               eta_r_h: Optional[np.ndarray] = None) -> dict:
    out = {
        "status": STATUS.get(info.status, info.status),
        "iters": info.iters,
        "outer_iters": info.outer_iters,
        "matvecs": info.matvecs,
        "rel_res_true": info.rel_res_true,
        "rel_res": info.rel_res,
        "eta_r": info.eta_r,
        "eta_e": info.eta_e,
        "launches": info.launches,
        "ct_plans": [n for bit, n in CT_PLANS.items() if info.ct_plans & bit],
    }
    if hist is not None:
        out["history"] = hist[: info.history_len].copy()
    if eta_e_h is not None:
        out["eta_e_history"] = eta_e_h[: info.eta_e_len].copy()
    if eta_r_h is not None:
        out["eta_r_history"] = eta_r_h[: info.eta_r_len].copy()
    return out


class Solver:
    """One microstructure on one grid (fh_create ... fh_destroy).

    phase      uint8 image of shape N (numpy on the host, or a CUDA torch tensor)
    L          per-phase tensors, shape (nphase, d, d), float64
    L0         reference conductivity (d, d) or None for Eq. (opt_ref)
    Y          cell half sizes (d,) or None
    precision  "fp64", "fp32" or "fp32_refined"
    """

    def __init__(self, phase, L, L0=None, Y=None, precision: str = "fp64", stream=None):
        import torch

        self._torch = torch
        self.lib = load_library()
        if torch.is_tensor(phase):
            on_dev = phase.is_cuda
            N = tuple(phase.shape)
            ph_ptr = phase.data_ptr()
            self._phase_ref = phase
        else:
            ph = np.ascontiguousarray(phase, dtype=np.uint8)
            on_dev = False
            N = ph.shape
            ph_ptr = ph.ctypes.data
            self._phase_ref = ph
        self.N = tuple(int(n) for n in N)
        self.d = len(self.N)
        Lh = np.ascontiguousarray(L, dtype=np.float64)
        self.nphase = Lh.shape[0]
        L0h = None if L0 is None else np.ascontiguousarray(L0, dtype=np.float64)
        Yh = None if Y is None else np.ascontiguousarray(Y, dtype=np.float64)
        Nh = (ctypes.c_int * self.d)(*self.N)
        self.precision = precision
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.dev = torch.device("cuda", torch.cuda.current_device())
        ctx = ctypes.c_void_p()
        rc = self.lib.fh_create(ctypes.byref(ctx), self.d, Nh,
                                None if Yh is None else _dptr(Yh),
                                ctypes.c_void_p(ph_ptr), int(on_dev), self.nphase, _dptr(Lh),
                                None if L0h is None else _dptr(L0h), PRECISIONS[precision],
                                ctypes.c_void_p(stream.cuda_stream))
        if rc != FH_OK:
            raise FhError(rc, "fh_create failed")
        self.ctx = ctx

    # -- lifecycle --------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.fh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc: int, what: str):
        if rc != FH_OK:
            raise FhError(rc, f"{what}: {self.lib.fh_last_error(self.ctx).decode()}")

    # -- calls ------------------------------------------------------------
    def set_phase(self, phase):
        torch = self._torch
        if torch.is_tensor(phase):
            rc = self.lib.fh_set_phase(self.ctx, ctypes.c_void_p(phase.data_ptr()), int(phase.is_cuda))
        else:
            ph = np.ascontiguousarray(phase, dtype=np.uint8)
            rc = self.lib.fh_set_phase(self.ctx, ctypes.c_void_p(ph.ctypes.data), 0)
        self._check(rc, "fh_set_phase")

    def apply(self, e, out=None, transpose: bool = False):
        """(I + B) e or (I + B^T) e for a CUDA tensor e of shape (d, *N)."""
        torch = self._torch
        assert e.is_cuda and e.is_contiguous() and tuple(e.shape) == (self.d,) + self.N
        dt = DT_FP64 if e.dtype == torch.float64 else DT_FP32
        if out is None:
            out = torch.empty_like(e)
        rc = self.lib.fh_apply(self.ctx, ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                               int(transpose), dt)
        self._check(rc, "fh_apply")
        return out

    def solve(self, E: Sequence[float], tol: float = 1e-8, method: str = "cg", max_iter: int = 10000,
              e_init=None, out=None, history: int = 0, want_field: bool = True, check: bool = False,
              eta_e: bool = False, norms: bool = False):
        """Solve for the load E.  Returns (field or None, L_eff column, info dict);
        info["eta_e"] is computed (one float64 pass) only when eta_e is true.
        With history > 0 and norms true, info["eta_e_history"] and
        info["eta_r_history"] hold Eq. (errE_def) of every iterate and
        Eq. (errR_def) of every step (FH_FP64 and FH_FP32 contexts)."""
        torch = self._torch
        Eh = np.ascontiguousarray(E, dtype=np.float64)
        if want_field and out is None:
            out = torch.empty((self.d,) + self.N, dtype=torch.float64, device=self.dev)
        col = np.zeros(self.d)
        info = FhInfo()
        info.flags = 1 if eta_e else 0
        hist = eh = rh = None
        if history > 0:
            hist = np.zeros(history)
            info.history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            info.history_cap = history
            if norms:
                eh, rh = np.zeros(history), np.zeros(history)
                info.eta_e_history = eh.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                info.eta_r_history = rh.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        rc = self.lib.fh_solve(self.ctx, _dptr(Eh), float(tol), METHODS[method], int(max_iter),
                               None if e_init is None else ctypes.c_void_p(e_init.data_ptr()),
                               None if out is None else ctypes.c_void_p(out.data_ptr()),
                               _dptr(col), ctypes.byref(info))
        if check:
            self._check(rc, "fh_solve")
        elif rc not in (FH_OK, 6, 7):
            self._check(rc, "fh_solve")
        return out, col, _info_dict(info, hist, eh, rh)

    def solve_all(self, tol: float = 1e-8, method: str = "cg", max_iter: int = 10000):
        Leff = np.zeros((self.d, self.d))
        infos = (FhInfo * self.d)()
        rc = self.lib.fh_solve_all(self.ctx, float(tol), METHODS[method], int(max_iter), _dptr(Leff), infos)
        if rc not in (FH_OK, 6, 7):
            self._check(rc, "fh_solve_all")
        return Leff, [_info_dict(infos[i], None) for i in range(self.d)]

    def profile(self, what: int, reps: int = 20, dtype: str = "fp32") -> float:
        """Average ms per launch of one piece of the CG iteration (fh_profile)."""
        v = np.zeros(1)
        self._check(self.lib.fh_profile(self.ctx, DT_FP64 if dtype == "fp64" else DT_FP32, int(what),
                                        int(reps), _dptr(v)), "fh_profile")
        return float(v[0])

    def autotune(self, dtype: str = "fp32", loads: bool = False):
        """Pick the fastest launch shapes (fh_autotune, or fh_autotune_loads for the
        all-loads pipeline of solve_all); returns (ms_before, ms_after)."""
        b, a = np.zeros(1), np.zeros(1)
        if loads:
            self._check(self.lib.fh_autotune_loads(self.ctx, _dptr(b), _dptr(a)), "fh_autotune_loads")
        else:
            self._check(self.lib.fh_autotune(self.ctx, DT_FP64 if dtype == "fp64" else DT_FP32, _dptr(b),
                                             _dptr(a)), "fh_autotune")
        return float(b[0]), float(a[0])

    def project_compatible(self, f, out=None):
        """Q f: the compatible part of a float64 field (fh_project_compatible)."""
        if out is None:
            out = self._torch.empty_like(f)
        self._check(self.lib.fh_project_compatible(self.ctx, ctypes.c_void_p(f.data_ptr()),
                                                   ctypes.c_void_p(out.data_ptr())), "fh_project_compatible")
        return out

    def effective_column(self, e) -> np.ndarray:
        col = np.zeros(self.d)
        self._check(self.lib.fh_effective_column(self.ctx, ctypes.c_void_p(e.data_ptr()), _dptr(col)),
                    "fh_effective_column")
        return col

    def eta_e(self, e) -> float:
        v = np.zeros(1)
        self._check(self.lib.fh_eta_e(self.ctx, ctypes.c_void_p(e.data_ptr()), _dptr(v)), "fh_eta_e")
        return float(v[0])


class Batch:
    """Independent 2-D cells of (possibly) different sizes solved together
    (fh_batch_create / fh_batch_solve / fh_batch_destroy).

    phases   list of uint8 images (each 2-D, odd sizes)
    tables   list of per-phase tensor tables, each (nphase, 2, 2)
    """

    def __init__(self, phases, tables, nloads: int = 2, precision: str = "fp32_refined"):
        self.lib = load_library()
        self.n = len(phases)
        self.nloads = nloads
        self._ph = [np.ascontiguousarray(p, dtype=np.uint8) for p in phases]
        self._L = [np.ascontiguousarray(t, dtype=np.float64) for t in tables]
        N = np.array([s for p in self._ph for s in p.shape], dtype=np.int32)
        nph = np.array([t.shape[0] for t in self._L], dtype=np.int32)
        php = (ctypes.c_void_p * self.n)(*[p.ctypes.data for p in self._ph])
        Lp = (ctypes.c_void_p * self.n)(*[t.ctypes.data for t in self._L])
        b = ctypes.c_void_p()
        rc = self.lib.fh_batch_create(ctypes.byref(b), self.n, N.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      php, nph.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), Lp, nloads,
                                      PRECISIONS[precision])
        if rc != FH_OK:
            raise FhError(rc, "fh_batch_create failed")
        self.b = b

    def autotune(self):
        """Tune every size group's launch shapes (fh_batch_autotune); returns
        (ms_before, ms_after), the summed CG-iteration time of all groups."""
        bf, af = np.zeros(1), np.zeros(1)
        rc = self.lib.fh_batch_autotune(self.b, _dptr(bf), _dptr(af))
        if rc != FH_OK:
            raise FhError(rc, "fh_batch_autotune: " + self.lib.fh_batch_last_error(self.b).decode())
        return float(bf[0]), float(af[0])

    def solve(self, E, tol: float = 1e-6, method: str = "cg", max_iter: int = 20000):
        """Returns (Leff [ncells, 2, nloads], status [ncells, nloads], iters, summary)."""
        Eh = np.ascontiguousarray(E, dtype=np.float64).reshape(-1)
        Leff = np.zeros((self.n, 2, self.nloads))
        st = np.zeros((self.n, self.nloads), dtype=np.int32)
        it = np.zeros((self.n, self.nloads), dtype=np.int32)
        info = FhInfo()
        rc = self.lib.fh_batch_solve(self.b, _dptr(Eh), float(tol), METHODS[method], int(max_iter), _dptr(Leff),
                                     st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                     it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(info))
        if rc not in (FH_OK, 6, 7):
            raise FhError(rc, self.lib.fh_batch_last_error(self.b).decode())
        return Leff, st, it, _info_dict(info, None)

    def close(self):
        if getattr(self, "b", None):
            self.lib.fh_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Net:
    """The warm-start network (fh_nn_*): float32 activations, bfloat16 weights.

    N        grid (3 ints, multiples of 27); cin / cout channels;
    channels (c0, c1, c2, c3) or None for (16, 32, 48, 64).
    """

    def __init__(self, N, cin: int, cout: int, channels=None, stream=None):
        import torch

        self._torch = torch
        self.lib = load_library()
        self.N = tuple(int(n) for n in N)
        self.cin, self.cout = cin, cout
        Nh = (ctypes.c_int * 3)(*self.N)
        ch = None if channels is None else (ctypes.c_int * 4)(*channels)
        st = 0 if stream is None else stream.cuda_stream
        h = ctypes.c_void_p()
        rc = self.lib.fh_nn_create(ctypes.byref(h), Nh, cin, cout, ch, ctypes.c_void_p(st))
        if rc != FH_OK:
            raise FhError(rc, "fh_nn_create failed")
        self.h = h
        self.nparam = int(self.lib.fh_nn_param_count(h))
        self.step = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.fh_nn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc, what):
        if rc != FH_OK:
            raise FhError(rc, what)

    def set_params(self, flat: np.ndarray):
        f = np.ascontiguousarray(flat, dtype=np.float32)
        self._chk(self.lib.fh_nn_set_params(self.h, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), f.size),
                  "fh_nn_set_params")
        self.step = 0

    def get_params(self) -> np.ndarray:
        f = np.zeros(self.nparam, dtype=np.float32)
        self._chk(self.lib.fh_nn_get_params(self.h, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), f.size),
                  "fh_nn_get_params")
        return f

    def forward(self, x, out=None):
        torch = self._torch
        if out is None:
            out = torch.empty((self.cout,) + self.N, dtype=torch.float32, device=x.device)
        self._chk(self.lib.fh_nn_forward(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr())),
                  "fh_nn_forward")
        return out

    def gradients(self, x, target):
        g = np.zeros(self.nparam, dtype=np.float32)
        loss = np.zeros(1)
        self._chk(self.lib.fh_nn_gradients(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                           _dptr(loss), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                  "fh_nn_gradients")
        return float(loss[0]), g

    def train_step(self, x, target, lr: float) -> float:
        self.step += 1
        loss = np.zeros(1)
        self._chk(self.lib.fh_nn_train_step(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                            float(lr), self.step, _dptr(loss)), "fh_nn_train_step")
        return float(loss[0])

    def launches(self) -> int:
        return int(self.lib.fh_nn_launches(self.h))


def nn_features(phase_dev, L, out):
    """Network input (2 channels) from a device phase image and its isotropic table."""
    lib = load_library()
    Lh = np.ascontiguousarray(L, dtype=np.float64)
    rc = lib.fh_nn_features(ctypes.c_void_p(phase_dev.data_ptr()), Lh.shape[0], _dptr(Lh), Lh.shape[-1],
                            phase_dev.numel(), ctypes.c_void_p(out.data_ptr()), None)
    if rc != FH_OK:
        raise FhError(rc, "fh_nn_features")
    return out


def nn_response_features(solver: "Solver", out):
    """out[b*d + a] = (B e_b)_a, float32 [d*d][N...] on the device."""
    lib = load_library()
    rc = lib.fh_nn_response_features(solver.ctx, solver.d, int(np.prod(solver.N)), ctypes.c_void_p(out.data_ptr()))
    if rc != FH_OK:
        raise FhError(rc, "fh_nn_response_features")
    return out


def nn_targets(fields, out, base=None):
    """Training target (d*d channels) from the d solved unit-load fields (float64,
    device), measured from base (float32 [d*d][N...] or None)."""
    lib = load_library()
    d = len(fields)
    arr = (ctypes.c_void_p * d)(*[f.data_ptr() for f in fields])
    nodes = fields[0].numel() // d
    rc = lib.fh_nn_targets(arr, d, nodes, None if base is None else ctypes.c_void_p(base.data_ptr()),
                           ctypes.c_void_p(out.data_ptr()), None)
    if rc != FH_OK:
        raise FhError(rc, "fh_nn_targets")
    return out


def nn_warm_start(solver: "Solver", pred, E, out, base=None):
    """x0 = E + Q(sum_b E_b (pred_b - base_b)): the projected warm start for load E."""
    lib = load_library()
    Eh = np.ascontiguousarray(E, dtype=np.float64)
    nodes = int(np.prod(solver.N))
    rc = lib.fh_nn_warm_start(solver.ctx, ctypes.c_void_p(pred.data_ptr()),
                              None if base is None else ctypes.c_void_p(base.data_ptr()), _dptr(Eh), solver.d,
                              nodes, ctypes.c_void_p(out.data_ptr()), None)
    if rc != FH_OK:
        raise FhError(rc, "fh_nn_warm_start")
    return out


def set_wait_limit(seconds: float) -> None:
    """Limit of the bounded device waits (fh_set_wait_limit); 0 = default 2 s."""
    rc = load_library().fh_set_wait_limit(float(seconds))
    if rc != FH_OK:
        raise FhError(rc, "fh_set_wait_limit")


def wait_selftest(seconds: float, stream=None) -> int:
    """fh_wait_selftest: the status of one bounded wait that nothing completes."""
    st = 0 if stream is None else stream.cuda_stream
    return int(load_library().fh_wait_selftest(float(seconds), ctypes.c_void_p(st)))


def version() -> str:
    return load_library().fh_version().decode()
