"""GB300 (sm_103a) recursive Fermi-operator expansion: D = f(Hp), tr(Hp D).

Thin ctypes binding of the C ABI in ``include/fe.h`` / ``include/fe_kernels.h``.
It only marshals arguments (pointers, sizes, flags); every step of the solve
runs in the library's CUDA kernels.  PyTorch, when used, only provides device
memory and the current stream.  There is no CPU fallback: if the library or a
GB300 is missing, the calls raise.
"""
import ctypes
import os

import numpy as np

from . import build as _build

FE_OK, FE_PENDING, FE_EINVAL, FE_ENOMEM, FE_ENOTCONV, FE_ETIMEOUT, FE_ECUDA, FE_EBUSY = (
    0, 1, -1, -2, -3, -4, -5, -6)
STATUS_NAMES = {0: "FE_OK", 1: "FE_PENDING", -1: "FE_EINVAL", -2: "FE_ENOMEM", -3: "FE_ENOTCONV",
                -4: "FE_ETIMEOUT", -5: "FE_ECUDA", -6: "FE_EBUSY"}
FE_PTR_HOST, FE_PTR_DEVICE = 0x0, 0x1
FE_METHOD_AUTO, FE_METHOD_SP2, FE_METHOD_FERMI, FE_METHOD_ASP2, FE_METHOD_TRFOE = 0x00, 0x10, 0x20, 0x30, 0x40
PREC = {"mixed": 0x000, "fp64": 0x100, "fp32": 0x200, "try_fp16": 0x300}


class FeConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t),
                ("max_iters", ctypes.c_int), ("precision_policy", ctypes.c_uint32),
                ("cuda_stream", ctypes.c_void_p), ("autotune_path", ctypes.c_char_p)]


class FeProblem(ctypes.Structure):
    _fields_ = [("Hp", ctypes.c_void_p), ("n", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("n_e", ctypes.c_double), ("kT", ctypes.c_double), ("tol", ctypes.c_double),
                ("D", ctypes.c_void_p), ("flags", ctypes.c_uint32), ("homo", ctypes.c_double),
                ("lumo", ctypes.c_double)]


class FeTune(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("bn", ctypes.c_int), ("ms_256", ctypes.c_double),
                ("ms_128", ctypes.c_double)]


class FeResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("iters_by_phase", ctypes.c_int * 4), ("e_band", ctypes.c_double),
                ("trace", ctypes.c_double), ("idem_fro", ctypes.c_double), ("mu", ctypes.c_double),
                ("eps_min", ctypes.c_double), ("eps_max", ctypes.c_double), ("ms", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "iters_by_phase"}
        d["iters_by_phase"] = list(self.iters_by_phase)
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


_lib = None


def lib_path():
    return _build.LIB


def load(build=True):
    """Load (building first if needed) libfe.so and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, dbl = ctypes.c_int64, ctypes.c_double
    L.fe_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(FeConfig)]
    L.fe_destroy.argtypes = [P]
    L.fe_solve.argtypes = [P, ctypes.POINTER(FeProblem), ctypes.POINTER(FeResult)]
    L.fe_solve_batch.argtypes = [P, ctypes.c_int, ctypes.POINTER(FeProblem), ctypes.POINTER(FeResult)]
    L.fe_submit.argtypes = [P, ctypes.POINTER(FeProblem), ctypes.POINTER(ctypes.c_uint64)]
    L.fe_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(FeResult)]
    L.fe_last_error_string.argtypes = [P]
    L.fe_last_error_string.restype = ctypes.c_char_p
    L.fe_k_gershgorin.argtypes = [P, P, i64, i64, ctypes.POINTER(dbl)]
    L.fe_project.argtypes = [P, P, P, i64, i64, i64, P, i64]
    L.fe_rotate.argtypes = [P, P, i64, i64, i64, P, i64, P, i64]
    L.fe_k_sym_square.argtypes = [P, P, i64, i64, P, i64, ctypes.c_int, dbl]
    L.fe_k_gershgorin_noalloc.argtypes = [P, i64, i64, P, P]
    L.fe_k_digit_square.argtypes = [P, P, i64, i64, P, i64]
    L.fe_k_profile.argtypes = [P, ctypes.c_int]
    L.fe_k_narrow_bounds.argtypes = [P, dbl]
    L.fe_k_set_wait.argtypes = [P, dbl, ctypes.c_int]
    L.fe_k_serve_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.c_int]
    L.fe_k_profile_kinds.argtypes = [P, ctypes.POINTER(dbl), ctypes.POINTER(ctypes.c_int)]
    L.fe_k_phase_ms.argtypes = [P, ctypes.POINTER(dbl)]
    L.fe_k_profile_steps.argtypes = [P, ctypes.POINTER(dbl), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.fe_k_profile_read.argtypes = [P, ctypes.POINTER(dbl)]
    L.fe_k_launch_count.argtypes = [P, ctypes.POINTER(i64)]
    L.fe_k_history.argtypes = [P, ctypes.c_int, ctypes.POINTER(dbl), ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int)]
    L.fe_autotune.argtypes = [P, ctypes.c_int, ctypes.POINTER(i64), ctypes.c_uint32, ctypes.c_int,
                              ctypes.POINTER(FeTune)]
    L.fe_autotune_batch.argtypes = [P, ctypes.c_int, ctypes.POINTER(FeProblem), ctypes.c_int,
                                    ctypes.POINTER(dbl), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.fe_k_set_tile_width.argtypes = [P, i64, ctypes.c_uint32, ctypes.c_int]
    L.fe_k_tile_width.argtypes = [P, i64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int)]
    for name in ("fe_create", "fe_destroy", "fe_solve", "fe_solve_batch", "fe_submit", "fe_poll",
                 "fe_project", "fe_rotate",
                 "fe_k_gershgorin", "fe_k_gershgorin_noalloc", "fe_k_sym_square", "fe_k_digit_square",
                 "fe_k_profile", "fe_k_profile_read", "fe_k_narrow_bounds", "fe_k_set_wait", "fe_k_serve_stats", "fe_k_profile_kinds", "fe_k_phase_ms",
                 "fe_k_profile_steps",
                 "fe_k_launch_count", "fe_k_history", "fe_autotune", "fe_autotune_batch", "fe_k_set_tile_width",
                 "fe_k_tile_width"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class FeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _ptr(x):
    """(address, is_device, keepalive) of a torch tensor or numpy array."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data, False, x
    import torch
    if isinstance(x, torch.Tensor):
        return x.data_ptr(), x.is_cuda, x
    raise TypeError("expected a numpy array or torch tensor")


def _ready(*xs):
    """A context runs on its own non-blocking stream, which is not ordered
    after torch's: wait until torch's current stream has written the device
    tensors handed to the library."""
    import sys
    torch = sys.modules.get("torch")
    if torch is None:
        return
    for x in xs:
        if isinstance(x, torch.Tensor) and x.is_cuda:
            torch.cuda.current_stream(x.device).synchronize()
            return


def gershgorin_noalloc(H, out4, stream=None):
    """Gershgorin bounds of a device FP64 matrix H into the device tensor out4
    (4 doubles), through the entry point that allocates nothing and needs no
    context (for callers whose memory is owned by their own pool, or who must
    not trigger cudaMalloc's device-wide synchronisation).  Queued on `stream`
    (a raw cudaStream_t; default: torch's current stream) without waiting.
    Calls that overlap in time share one scratch array and race."""
    import torch
    L = load()
    if not (isinstance(H, torch.Tensor) and isinstance(out4, torch.Tensor)):
        raise ValueError("torch tensors expected")
    dev = torch.cuda.current_device()
    if not (H.is_cuda and out4.is_cuda and H.device.index == dev and out4.device.index == dev):
        raise ValueError("H and out4 must be on the current CUDA device")
    if H.dtype != torch.float64 or H.dim() != 2 or H.shape[0] != H.shape[1] or H.stride(1) != 1:
        raise ValueError("H must be a square float64 matrix with unit column stride")
    if out4.dtype != torch.float64 or out4.numel() < 4 or not out4.is_contiguous():
        raise ValueError("out4 must be a contiguous float64 tensor of at least 4 elements")
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    rc = L.fe_k_gershgorin_noalloc(H.data_ptr(), H.shape[0], H.stride(0), out4.data_ptr(),
                                   ctypes.c_void_p(stream))
    if rc != FE_OK:
        raise FeError(rc, L.fe_last_error_string(None).decode())


class Context:
    """One library context (fe_create) on one GPU."""

    def __init__(self, device=0, hbm_budget_bytes=0, max_iters=0, precision="mixed", stream=None,
                 autotune_path=None):
        self.L = load()
        cfg = FeConfig(device, hbm_budget_bytes, max_iters, PREC[precision],
                       ctypes.c_void_p(stream) if stream else None,
                       os.fsencode(autotune_path) if autotune_path else None)
        h = ctypes.c_void_p()
        rc = self.L.fe_create(ctypes.byref(h), ctypes.byref(cfg))
        if rc != FE_OK:
            raise FeError(rc, self.L.fe_last_error_string(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.fe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def last_error(self):
        return self.L.fe_last_error_string(self.h).decode()

    def _problem(self, H, ne, kT, tol, D, precision, method, homo=0.0, lumo=0.0):
        hp, hdev, keep_h = _ptr(H)
        n = H.shape[0]
        assert H.shape[0] == H.shape[1]
        ld = (H.stride(0) if hasattr(H, "stride") and callable(H.stride) else H.strides[0] // 8)
        dp = None
        keep_d = None
        if D is not None:
            dp, ddev, keep_d = _ptr(D)
            if ddev != hdev:
                raise ValueError("Hp and D must both be host or both be device buffers")
            dld = (D.stride(0) if hasattr(D, "stride") and callable(D.stride) else D.strides[0] // 8)
            if dld != ld:
                raise ValueError("Hp and D must share the leading dimension")
        flags = (FE_PTR_DEVICE if hdev else FE_PTR_HOST) | PREC[precision] | method
        p = FeProblem(hp, n, ld, float(ne), float(kT), float(tol), dp, flags, float(homo), float(lumo))
        _ready(H, D)
        return p, (keep_h, keep_d)

    def solve(self, H, ne, kT=0.0, tol=0.0, D=None, precision="mixed", method=FE_METHOD_AUTO,
              check=True, homo=0.0, lumo=0.0):
        """Solve one problem.  H (n x n FP64, host numpy or device torch); D
        (same kind, written) or None; homo/lumo: the HOMO/LUMO estimates of
        FE_METHOD_ASP2.  Returns the result dict."""
        p, keep = self._problem(H, ne, kT, tol, D, precision, method, homo, lumo)
        r = FeResult()
        rc = self.L.fe_solve(self.h, ctypes.byref(p), ctypes.byref(r))
        if check and rc != FE_OK:
            raise FeError(rc, self.last_error())
        out = r.as_dict()
        out["rc"] = rc
        return out

    def solve_batch(self, items, check=True):
        """items: list of dict(H=..., ne=..., kT=0, tol=0, D=None, precision='mixed')."""
        probs = (FeProblem * len(items))()
        keep = []
        for k, it in enumerate(items):
            p, kp = self._problem(it["H"], it["ne"], it.get("kT", 0.0), it.get("tol", 0.0),
                                  it.get("D"), it.get("precision", "mixed"),
                                  it.get("method", FE_METHOD_AUTO), it.get("homo", 0.0), it.get("lumo", 0.0))
            probs[k] = p
            keep.append(kp)
        res = (FeResult * len(items))()
        rc = self.L.fe_solve_batch(self.h, len(items), probs, res)
        if check and rc != FE_OK:
            raise FeError(rc, self.last_error())
        return rc, [r.as_dict() for r in res]

    # ---- continuous batching -------------------------------------------------
    def submit(self, H, ne, kT=0.0, tol=0.0, D=None, precision="mixed", method=FE_METHOD_AUTO,
               homo=0.0, lumo=0.0):
        """Queue one problem; returns its ticket.  H may be reused at once; D
        (if given) must stay alive until poll() returns a final status."""
        p, keep = self._problem(H, ne, kT, tol, D, precision, method, homo, lumo)
        t = ctypes.c_uint64()
        rc = self.L.fe_submit(self.h, ctypes.byref(p), ctypes.byref(t))
        if rc != FE_OK:
            raise FeError(rc, self.last_error())
        self._keep = getattr(self, "_keep", {})
        self._keep[t.value] = keep[1]
        return t.value

    def poll(self, ticket):
        """None while pending; else the result dict (with 'rc')."""
        r = FeResult()
        rc = self.L.fe_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(r))
        if rc == FE_PENDING:
            return None
        if rc == FE_EINVAL and r.status == 0:
            raise FeError(rc, self.last_error())
        getattr(self, "_keep", {}).pop(ticket, None)
        out = r.as_dict()
        out["rc"] = rc
        return out

    def wait(self, ticket, timeout_s=600.0, sleep_s=0.0005):
        import time
        t0 = time.time()
        while True:
            res = self.poll(ticket)
            if res is not None:
                return res
            if time.time() - t0 > timeout_s:
                raise TimeoutError("ticket %d still pending" % ticket)
            time.sleep(sleep_s)

    # ---- either side of the expansion (device buffers) ------------------------
    def project(self, Psi, HPsi, Hp):
        """Hp = Psi^T HPsi (Rayleigh-Ritz projection): Psi, HPsi m x n, Hp n x n,
        FP64 device tensors with unit column stride."""
        for t in (Psi, HPsi, Hp):
            if not (getattr(t, "is_cuda", False) and t.stride(1) == 1):
                raise ValueError("device tensors with unit column stride expected")
        if HPsi.shape != Psi.shape or HPsi.stride(0) != Psi.stride(0):
            raise ValueError("Psi and HPsi must have the same shape and leading dimension")
        m, n = Psi.shape
        _ready(Psi, HPsi, Hp)
        rc = self.L.fe_project(self.h, Psi.data_ptr(), HPsi.data_ptr(), m, n, Psi.stride(0), Hp.data_ptr(),
                               Hp.stride(0))
        if rc != FE_OK:
            raise FeError(rc, self.last_error())

    def rotate(self, Psi, D, Out):
        """Out = Psi D for a symmetric D (subspace rotation / density): Psi and
        Out m x n, D n x n, FP64 device tensors with unit column stride."""
        for t in (Psi, D, Out):
            if not (getattr(t, "is_cuda", False) and t.stride(1) == 1):
                raise ValueError("device tensors with unit column stride expected")
        m, n = Psi.shape
        _ready(Psi, D, Out)
        rc = self.L.fe_rotate(self.h, Psi.data_ptr(), m, n, Psi.stride(0), D.data_ptr(), D.stride(0),
                              Out.data_ptr(), Out.stride(0))
        if rc != FE_OK:
            raise FeError(rc, self.last_error())

    # ---- single kernels (device buffers) -------------------------------------
    def gershgorin(self, H):
        hp, hdev, _ = _ptr(H)
        assert hdev, "device tensor expected"
        out = (ctypes.c_double * 4)()
        _ready(H)
        rc = self.L.fe_k_gershgorin(self.h, hp, H.shape[0], H.stride(0), out)
        if rc != FE_OK:
            raise FeError(rc, self.last_error())
        return list(out)

    def sym_square(self, Y, C, nslices=2, bound=None):
        yp, ydev, _ = _ptr(Y)
        cp, cdev, _ = _ptr(C)
        assert ydev and cdev, "device tensors expected"
        if bound is None:
            bound = float(Y.abs().max())
        _ready(Y, C)
        rc = self.L.fe_k_sym_square(self.h, yp, Y.shape[0], Y.stride(0), cp, C.stride(0),
                                    int(nslices), float(bound))
        if rc != FE_OK:
            raise FeError(rc, self.last_error())

    def digit_square(self, X, P):
        """P = X @ X (FP64 device tensors) by the FP64-accurate digit kernel."""
        xp, xdev, _ = _ptr(X)
        pp, pdev, _ = _ptr(P)
        assert xdev and pdev, "device tensors expected"
        _ready(X, P)
        rc = self.L.fe_k_digit_square(self.h, xp, X.shape[0], X.stride(0), pp, P.stride(0))
        if rc != FE_OK:
            raise FeError(rc, self.last_error())

    # ---- tile-shape autotuner ---------------------------------------------------
    def autotune(self, ns, precision="mixed", reps=2):
        """Time synthetic solves of each size in `ns` with 128 x 256 and
        128 x 128 tensor-core tiles and keep the faster width per size
        (fe_autotune); returns one dict per size."""
        ns = [int(x) for x in ns]
        arr = (ctypes.c_int64 * max(1, len(ns)))(*ns)
        out = (FeTune * max(1, len(ns)))()
        rc = self.L.fe_autotune(self.h, len(ns), arr, PREC[precision], int(reps), out)
        if rc != FE_OK:
            raise FeError(rc, self.last_error())
        return [{"n": t.n, "bn": t.bn, "ms_256": t.ms_256, "ms_128": t.ms_128} for t in out[: len(ns)]]

    def autotune_batch(self, items, reps=2, max_trials=64):
        """Tune the tile widths on a batch (fe_autotune_batch; items as for
        solve_batch, outputs not written).  Returns the trials' batch times
        (ms; the first with 128 x 256 tiles everywhere)."""
        probs = (FeProblem * len(items))()
        keep = []
        for k, it in enumerate(items):
            p, kp = self._problem(it["H"], it["ne"], it.get("kT", 0.0), it.get("tol", 0.0), None,
                                  it.get("precision", "mixed"), it.get("method", FE_METHOD_AUTO))
            probs[k] = p
            keep.append(kp)
        out = (ctypes.c_double * max_trials)()
        nt = ctypes.c_int()
        rc = self.L.fe_autotune_batch(self.h, len(items), probs, int(reps), out, int(max_trials),
                                      ctypes.byref(nt))
        if rc != FE_OK:
            raise FeError(rc, self.last_error())
        return list(out[: min(nt.value, max_trials)])

    def set_tile_width(self, n, bn, precision="mixed"):
        """Make problems with n's number of 128-row panels use tile width bn
        (128 or 256; 0 removes the entry)."""
        rc = self.L.fe_k_set_tile_width(self.h, int(n), PREC[precision], int(bn))
        if rc != FE_OK:
            raise FeError(rc, self.last_error())

    def tile_width(self, n, precision="mixed"):
        v = ctypes.c_int()
        rc = self.L.fe_k_tile_width(self.h, int(n), PREC[precision], ctypes.byref(v))
        if rc != FE_OK:
            raise FeError(rc, self.last_error())
        return v.value

    # ---- measurement hooks ----------------------------------------------------
    def profile(self, enable=True):
        self.L.fe_k_profile(self.h, 1 if enable else 0)

    def profile_read(self):
        out = (ctypes.c_double * 8)()
        self.L.fe_k_profile_read(self.h, out)
        keys = ("tc_ms", "tc_launches", "fp64_ms", "fp64_launches", "solve_ms", "launches_total",
                "tc_ms_all", "tc_launches_all")
        return dict(zip(keys, list(out)))

    def set_wait(self, limit_ms=2000.0, fail_partner=False):
        """Failure-detection hook: the limit of the kernels' bounded waits and
        the test word that makes the split-tile partner wait run out."""
        rc = self.L.fe_k_set_wait(self.h, float(limit_ms), 1 if fail_partner else 0)
        if rc != FE_OK:
            raise FeError(rc, self.last_error())

    def profile_kinds(self):
        """Step launches of the last profiled solve by kind: {name: (ms, launches)}."""
        ms = (ctypes.c_double * 8)()
        cnt = (ctypes.c_int * 8)()
        rc = self.L.fe_k_profile_kinds(self.h, ms, cnt)
        if rc != FE_OK:
            raise FeError(rc, self.last_error())
        names = {1: "single_fp16", 2: "split_fp16", 3: "fp64", 5: "epilogue_only", 6: "digit",
                 7: "polish_delta"}
        return {v: (ms[k], cnt[k]) for k, v in names.items()}

    def narrow_bounds(self, factor):
        """Test hook: shrink the estimated spectral bounds of later solves
        about their centre by `factor` (1 = off)."""
        rc = self.L.fe_k_narrow_bounds(self.h, float(factor))
        if rc != FE_OK:
            raise FeError(rc, self.last_error())

    def profile_steps(self, max_steps=400):
        """ms of each step's tensor-core launch in the last profiled solve."""
        out = (ctypes.c_double * max_steps)()
        cnt = ctypes.c_int()
        self.L.fe_k_profile_steps(self.h, out, int(max_steps), ctypes.byref(cnt))
        return list(out[: cnt.value])

    def phase_ms(self):
        """Device time of the last blocking solve by phase (CUDA events)."""
        out = (ctypes.c_double * 4)()
        self.L.fe_k_phase_ms(self.h, out)
        return dict(zip(("setup_ms", "loop_ms", "output_ms", "steps"), list(out)))

    def serve_stats(self, reset=False):
        """Serving counters: submitted, deferred (waited for HBM), peak
        waiting queue, peak requests on the device."""
        out = (ctypes.c_int64 * 4)()
        rc = self.L.fe_k_serve_stats(self.h, out, 1 if reset else 0)
        if rc != FE_OK:
            raise FeError(rc, self.last_error())
        return dict(zip(("submitted", "deferred", "peak_waiting", "peak_running"), list(out)))

    def launch_count(self):
        v = ctypes.c_int64()
        self.L.fe_k_launch_count(self.h, ctypes.byref(v))
        return v.value

    def history(self, index=0, max_rows=160):
        """Per-step record of the last solve (rows of phase, kind, t1-N_e,
        t1-t2, ||X^2-X||_F, RelTr)."""
        out = (ctypes.c_double * (6 * max_rows))()
        rows = ctypes.c_int()
        rc = self.L.fe_k_history(self.h, int(index), out, int(max_rows), ctypes.byref(rows))
        if rc != FE_OK:
            raise FeError(rc, self.last_error())
        return np.array(out[: 6 * rows.value]).reshape(rows.value, 6)
