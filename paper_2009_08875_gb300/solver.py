"""Python face of libst: argument marshalling between torch tensors and the C ABI."""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import STError  # noqa: F401


def _ptr(t, shape, name, device_ok=True, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != (dtype or torch.float64):
        raise TypeError(f"{name} must be {dtype or torch.float64}")
    if device_ok and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One handle of the CUDA solver for space level K and time level J on the unit square.

    Tensors are (N_t, N_x) float64 CUDA tensors; wavelet-coordinate tensors use the library's
    in-place row order.  Work is enqueued on `stream` (default: torch's current stream).
    """

    def __init__(self, K, J, domain=0, alpha=0.3, n_vcycles=2, n_pre=3, n_post=3, tol=1e-10, tol_mode=0,
                 maxit=200, precision="fp64", inner_tol=1e-5, inner_maxit=60, batch=1, use_graphs=2,
                 stream=None, D=None, c=0.0, initial_guess=False):
        import torch
        lib = _lib.load()
        cfg = _lib.StConfig()
        lib.st_default_config(ctypes.byref(cfg))
        cfg.alpha, cfg.n_vcycles, cfg.n_pre, cfg.n_post = alpha, n_vcycles, n_pre, n_post
        cfg.tol, cfg.tol_mode, cfg.maxit = tol, tol_mode, maxit
        cfg.precision = {"fp64": _lib.ST_FP64, "mixed": _lib.ST_MIXED_FP32,
                         "mixed_precond": _lib.ST_MIXED_PRECOND, "mixed_bf16": _lib.ST_MIXED_BF16,
                     "fp64_df": _lib.ST_FP64_DF}[precision]
        cfg.inner_tol, cfg.inner_maxit = inner_tol, inner_maxit
        cfg.use_graphs = int(use_graphs)  # 2: device-driven loop, 1: iteration-body graphs, 0: none
        cfg.initial_guess = 1 if initial_guess else 0
        _set_phys(cfg, D, c)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _lib.check(lib.st_setup_batch(ctypes.byref(h), domain, K, J, batch, ctypes.byref(cfg),
                                      ctypes.c_void_p(stream.cuda_stream)))
        self._h = h
        nt, nx = ctypes.c_int64(), ctypes.c_int64()
        _lib.check(lib.st_dims(h, ctypes.byref(nt), ctypes.byref(nx)))
        self.Nt, self.Nx = nt.value, nx.value
        self.K, self.J, self.B = K, J, batch

    @property
    def shape(self):
        """Shape of a space-time vector: (N_t, N_x), or (B, N_t, N_x) for a batch."""
        return (self.Nt, self.Nx) if self.B == 1 else (self.B, self.Nt, self.Nx)

    @property
    def u0_shape(self):
        return (self.Nx,) if self.B == 1 else (self.B, self.Nx)

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().st_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def apply_Kx(self, b, x):
        ns = b.shape[0]
        _lib.check(_lib.load().st_apply_Kx(self._h, ns, _ptr(b, (ns, self.Nx), "b"), _ptr(x, (ns, self.Nx), "x")))

    def apply_S_nodal(self, u, y):
        _lib.check(_lib.load().st_apply_S_nodal(self._h, _ptr(u, self.shape, "u"), _ptr(y, self.shape, "y")))

    def synthesize(self, w, u):
        _lib.check(_lib.load().st_synthesize(self._h, _ptr(w, self.shape, "w"), _ptr(u, self.shape, "u")))

    def analyze(self, u, w):
        _lib.check(_lib.load().st_analyze(self._h, _ptr(u, self.shape, "u"), _ptr(w, self.shape, "w")))

    def apply_S(self, w, q):
        _lib.check(_lib.load().st_apply_S(self._h, _ptr(w, self.shape, "w"), _ptr(q, self.shape, "q")))

    def apply_KX(self, r, z):
        _lib.check(_lib.load().st_apply_KX(self._h, _ptr(r, self.shape, "r"), _ptr(z, self.shape, "z")))

    def apply_S_f32(self, w, q):
        import torch
        _lib.check(_lib.load().st_apply_S_f32(self._h, _ptr(w, self.shape, "w", dtype=torch.float32),
                                              _ptr(q, self.shape, "q", dtype=torch.float32)))

    def apply_KX_f32(self, r, z):
        import torch
        _lib.check(_lib.load().st_apply_KX_f32(self._h, _ptr(r, self.shape, "r", dtype=torch.float32),
                                               _ptr(z, self.shape, "z", dtype=torch.float32)))

    def apply_KX_bf16(self, r, z):
        """K_X in binary32 arithmetic with bfloat16 multigrid storage (st_apply_KX_bf16)."""
        import torch
        _lib.check(_lib.load().st_apply_KX_bf16(self._h, _ptr(r, self.shape, "r", dtype=torch.float32),
                                                _ptr(z, self.shape, "z", dtype=torch.float32)))

    def solve_info(self):
        """Iterations, refinement steps and final relative residual of the last solve."""
        out = _lib.StSolveInfo()
        _lib.check(_lib.load().st_solve_info_get(self._h, ctypes.byref(out)))
        return {"iterations": out.iterations, "outer_iterations": out.outer_iterations, "relres": out.relres}

    def problem_info(self, b):
        """Iterations, refinement steps, final relative residual and status of problem b."""
        out, st = _lib.StSolveInfo(), ctypes.c_int()
        _lib.check(_lib.load().st_problem_info(self._h, b, ctypes.byref(out), ctypes.byref(st)))
        return {"iterations": out.iterations, "outer_iterations": out.outer_iterations, "relres": out.relres,
                "status": st.value}

    def rhs(self, g, u0, fhat):
        _lib.check(_lib.load().st_rhs(self._h, _ptr(g, self.shape, "g"), _ptr(u0, self.u0_shape, "u0"),
                                      _ptr(fhat, self.shape, "fhat")))

    def pcg_solve(self, fhat, w):
        it, rr = ctypes.c_int(), ctypes.c_double()
        st = _lib.load().st_pcg_solve(self._h, _ptr(fhat, self.shape, "fhat"), _ptr(w, self.shape, "w"),
                                      ctypes.byref(it), ctypes.byref(rr))
        if st not in (_lib.ST_OK,):
            _lib.check(st)
        return it.value, rr.value

    def solve_host(self, g, u0, u):
        """End-to-end solve from (preferably pinned) host tensors g (N_t, N_x), u0 (N_x,) into u."""
        it, rr = ctypes.c_int(), ctypes.c_double()
        st = _lib.load().st_solve_host(self._h, _ptr(g, self.shape, "g", False), _ptr(u0, self.u0_shape, "u0", False),
                                       _ptr(u, self.shape, "u", False), ctypes.byref(it), ctypes.byref(rr))
        _lib.check(st)
        return it.value, rr.value

    def nested_solve(self, levels, eps, g, u0, w, rate=1.0):
        """Nested iteration over (K - m, J - m), m = levels-1..0 (st_nested_solve): g, u0 nodal
        device tensors of this handle's mesh, w receives the finest solution (wavelet order).
        Returns (status, iterations per level, coarsest first)."""
        its = (ctypes.c_int * levels)()
        st = _lib.load().st_nested_solve(self._h, levels, eps, rate, _ptr(g, self.shape, "g"),
                                         _ptr(u0, self.u0_shape, "u0"), _ptr(w, self.shape, "w"), its)
        if st not in (0, _lib.ST_ERR_MAXIT):
            _lib.check(st)
        return st, list(its)

    def autotune(self):
        """Time the Gauss-Seidel kernels per level and keep the fastest (st_autotune).  Returns
        {level: {"f64_Kx": (tiles_ms, wave_ms, regs_ms), "f64_Kl": ..., "f32_Kx": ..., "f32_Kl": ...}}."""
        t = (ctypes.c_float * 192)()
        _lib.check(_lib.load().st_autotune(self._h, t))
        names = ("f64_Kx", "f64_Kl", "f32_Kx", "f32_Kl")
        return {k: {nm: (t[12 * k + 3 * i], t[12 * k + 3 * i + 1], t[12 * k + 3 * i + 2])
                    for i, nm in enumerate(names)}
                for k in range(2, self.K + 1) if any(t[12 * k + i] for i in range(12))}

    SMOOTHERS = {"tiles": 0, "wavefront": 1, "registers": 2, "registers_8x12": 3, "registers_6x16": 4,
                 "registers_wide": 5}

    def set_smoother(self, kind):
        """Force the Gauss-Seidel kernel on every level (st_set_smoother): 'tiles', 'wavefront',
        'registers' (12 rows x 8 warps in binary32), 'registers_8x12', 'registers_6x16', or the
        binary32 regions with paired arithmetic 'registers_wide' (192 or 96 columns; where a level
        holds no such region: 'registers')."""
        _lib.check(_lib.load().st_set_smoother(self._h, self.SMOOTHERS[kind]))

    def set_wave_rows(self, rows):
        """Rows per segment of the wavefront kernel on every level, 0 for the default (st_set_wave_rows)."""
        _lib.check(_lib.load().st_set_wave_rows(self._h, int(rows)))

    def profile_begin(self):
        """Start counting launches and timing finest-level sweeps (measurement hook)."""
        _lib.check(_lib.load().st_profile_begin(self._h))

    def profile_end(self):
        """Synchronise and return a dict with the launch count and the timed sweep totals."""
        out = _lib.StProfile()
        _lib.check(_lib.load().st_profile_end(self._h, ctypes.byref(out)))
        return {f: getattr(out, f) for f, _ in _lib.StProfile._fields_}


def _set_phys(cfg, D, c):
    """D (2 x 2 symmetric, or None for the identity) and c of the reaction-diffusion form."""
    if D is not None:
        cfg.diffusion[0], cfg.diffusion[1], cfg.diffusion[2] = float(D[0][0]), float(D[0][1]), float(D[1][1])
        if float(D[1][0]) != float(D[0][1]):
            raise ValueError("D must be symmetric")
    cfg.reaction = float(c)


def _config(alpha=0.3, n_vcycles=2, n_pre=3, n_post=3, tol=1e-10, tol_mode=0, maxit=200, precision="fp64",
            inner_tol=1e-5, inner_maxit=60, use_graphs=2, D=None, c=0.0):
    lib = _lib.load()
    cfg = _lib.StConfig()
    lib.st_default_config(ctypes.byref(cfg))
    cfg.alpha, cfg.n_vcycles, cfg.n_pre, cfg.n_post = alpha, n_vcycles, n_pre, n_post
    cfg.tol, cfg.tol_mode, cfg.maxit = tol, tol_mode, maxit
    cfg.precision = {"fp64": _lib.ST_FP64, "mixed": _lib.ST_MIXED_FP32,
                     "mixed_precond": _lib.ST_MIXED_PRECOND, "mixed_bf16": _lib.ST_MIXED_BF16,
                     "fp64_df": _lib.ST_FP64_DF}[precision]
    cfg.inner_tol, cfg.inner_maxit = inner_tol, inner_maxit
    cfg.use_graphs = int(use_graphs)
    _set_phys(cfg, D, c)
    return cfg


class Batch:
    """Many solves of any shape in one call (st_batch_*).  Inputs and outputs are host tensors
    (float64, contiguous; page-locked ones copy fastest) kept alive until run() returns."""

    def __init__(self, **cfg):
        self._cfg = _config(**cfg)
        h = ctypes.c_void_p()
        _lib.check(_lib.load().st_batch_create(ctypes.byref(h), ctypes.byref(self._cfg)))
        self._h = h
        self._keep = []

    def add(self, domain, K, J, g, u0, u):
        n = 2 ** K - 1
        Nt, Nx = 2 ** J + 1, (n ** 3 if domain == 2 else n * n)
        ids = ctypes.c_int()
        _lib.check(_lib.load().st_batch_add(self._h, domain, K, J, _ptr(g, (Nt, Nx), "g", False),
                                            _ptr(u0, (Nx,), "u0", False), _ptr(u, (Nt, Nx), "u", False),
                                            ctypes.byref(ids)))
        self._keep.append((g, u0, u))
        return ids.value

    def run(self):
        st = _lib.load().st_batch_run(self._h)
        if st not in (_lib.ST_OK, _lib.ST_ERR_MAXIT, _lib.ST_ERR_BREAKDOWN):
            _lib.check(st)
        return st

    def info(self, i):
        out, st = _lib.StSolveInfo(), ctypes.c_int()
        _lib.check(_lib.load().st_batch_problem_info(self._h, i, ctypes.byref(out), ctypes.byref(st)))
        return {"iterations": out.iterations, "outer_iterations": out.outer_iterations, "relres": out.relres,
                "status": st.value}

    def buckets(self):
        n = ctypes.c_int()
        _lib.check(_lib.load().st_batch_buckets(self._h, ctypes.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().st_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (st_server_*).  submit() takes host tensors that must stay
    alive until poll() reports the request done; stop() serves everything and shuts down."""

    QUEUED, RUNNING, DONE, FAILED = 0, 1, 2, 3

    def __init__(self, slots_per_group=16, memory_budget_gb=100.0, **cfg):
        cfg.setdefault("precision", "mixed_precond")
        self._cfg = _config(**cfg)
        h = ctypes.c_void_p()
        _lib.check(_lib.load().st_server_start(ctypes.byref(h), ctypes.byref(self._cfg), slots_per_group,
                                               memory_budget_gb))
        self._h = h
        self._keep = {}

    def submit(self, domain, K, J, g, u0, u, timeout=None):
        """Queue a solve; with timeout (seconds) it fails with ST_ERR_TIMEOUT if not done by then."""
        n = 2 ** K - 1
        Nt, Nx = 2 ** J + 1, (n ** 3 if domain == 2 else n * n)
        t = ctypes.c_int64()
        _lib.check(_lib.load().st_server_submit_deadline(self._h, domain, K, J, _ptr(g, (Nt, Nx), "g", False),
                                                         _ptr(u0, (Nx,), "u0", False),
                                                         _ptr(u, (Nt, Nx), "u", False),
                                                         float(timeout) if timeout else 0.0, ctypes.byref(t)))
        self._keep[t.value] = (g, u0, u)
        return t.value

    def cancel(self, ticket):
        _lib.check(_lib.load().st_server_cancel(self._h, ticket))

    def poll(self, ticket):
        st, status, info, lat = ctypes.c_int(), ctypes.c_int(), _lib.StSolveInfo(), ctypes.c_double()
        _lib.check(_lib.load().st_server_poll(self._h, ticket, ctypes.byref(st), ctypes.byref(status),
                                              ctypes.byref(info), ctypes.byref(lat)))
        if st.value >= self.DONE:
            self._keep.pop(ticket, None)
        return {"state": st.value, "status": status.value, "iterations": info.iterations, "relres": info.relres,
                "latency_s": lat.value}

    def stop(self):
        if getattr(self, "_h", None):
            h, self._h = self._h, None
            _lib.check(_lib.load().st_server_stop(h))

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def probe_fma_rates(stream=None):
    """The device's sustained fused multiply-add rates (st_probe_fma_rates): (binary64, binary32)
    fmas per second, measured on `stream` (default: torch's current stream)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    a, b = ctypes.c_double(), ctypes.c_double()
    _lib.check(_lib.load().st_probe_fma_rates(ctypes.c_void_p(st.cuda_stream), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value
