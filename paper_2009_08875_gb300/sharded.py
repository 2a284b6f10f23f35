"""Time-sharded Schur-complement PCG: the time axis split over ranks (the paper's Sec. 5.2 scheme).

Rank r of P owns the time rows [r m, (r + 1) m) of every space-time vector (m = 2^J / P, the last
rank also row 2^J), as an (nrows, N_x) tensor.  One PCG iteration then needs:

* the nodal rows of S (time mix, K_x, epilogue; Lemma 4.2): one neighbour row of U each side
  (the time matrices are tridiagonal), exchanged point to point;
* the wavelet transforms W, W^T (Eq. 3.1), which act along the whole time axis: the rows are
  exchanged into blocks of columns (an all-to-all), each rank lifts its columns over all N_t rows,
  and the result is exchanged back;
* K_X (Thm. 3.1), block diagonal in the wavelet rows: no communication;
* two inner products: a sum of the ranks' partial sums.

The arithmetic runs in the backend (`CudaBackend`: the C-ABI kernels of libst; the tests also
drive the same schedule with a CPU backend); the communication runs through a `Comm`
(`TorchComm`: torch.distributed, NCCL between GPUs or gloo on CPU).  Only the data path's real
exchanges are collectives; nothing else is replicated.
"""
from __future__ import annotations

import ctypes
import math

from . import _lib


# ----------------------------------------------------------------------------------------------
# partition
# ----------------------------------------------------------------------------------------------
def row_range(J: int, P: int, r: int):
    """[lo, hi) of the time rows of rank r (P a power of two, P <= 2^J)."""
    m = (1 << J) // P
    lo = r * m
    hi = lo + m + (1 if r == P - 1 else 0)
    return lo, hi


def col_range(Nx: int, P: int, r: int):
    return r * Nx // P, (r + 1) * Nx // P


def check_partition(J: int, P: int):
    if P < 1 or P & (P - 1) or P > (1 << J):
        raise ValueError("the number of ranks must be a power of two no larger than 2^J")


# ----------------------------------------------------------------------------------------------
# communication
# ----------------------------------------------------------------------------------------------
class TorchComm:
    """torch.distributed: point-to-point exchanges and a sum over ranks."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)
        self.cpu = dist.get_backend(group) == "gloo"

    def exchange(self, sends, recvs):
        """sends[s]: tensor for rank s; recvs[s]: buffer filled from rank s (self included)."""
        reqs = []
        for s, t in recvs.items():
            if s != self.rank:
                reqs.append(self.dist.irecv(t, src=self._global(s), group=self.group))
        for s, t in sends.items():
            if s != self.rank:
                reqs.append(self.dist.isend(t.contiguous(), dst=self._global(s), group=self.group))
        if self.rank in sends and self.rank in recvs:
            recvs[self.rank].copy_(sends[self.rank])
        for q in reqs:
            q.wait()

    def allreduce_sum(self, x: float) -> float:
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cpu" if self.cpu else "cuda")
        self.dist.all_reduce(t, group=self.group)
        return float(t.item())

    def _global(self, r):
        return r if self.group is None else self.dist.get_global_rank(self.group, r)


# ----------------------------------------------------------------------------------------------
# the CUDA backend: libst's row-block, column-block and vector entry points
# ----------------------------------------------------------------------------------------------
class CudaBackend:
    """Local operators of one rank on its rows (st_rows_*, st_wavelet_cols, st_vec_*), with a
    single-problem handle of the full mesh for coefficient tables and scratch."""

    def __init__(self, K, J, domain=0, **cfg):
        from .solver import Solver
        self.solver = Solver(K, J, domain=domain, **cfg)
        self.Nt, self.Nx, self.J = self.solver.Nt, self.solver.Nx, J
        self.lib = _lib.load()
        self.h = self.solver._h

    @staticmethod
    def _p(t):
        return ctypes.c_void_p(t.data_ptr())

    def empty(self, rows, cols):
        import torch
        return torch.empty((rows, cols), dtype=torch.float64, device="cuda")

    def zeros(self, rows, cols):
        import torch
        return torch.zeros((rows, cols), dtype=torch.float64, device="cuda")

    def nodal(self, mode, row0, u_halo, u_row0):
        y = self.empty(u_halo.shape[0] - 2, self.Nx)
        _lib.check(self.lib.st_rows_nodal(self.h, mode, row0, y.shape[0], self._p(u_halo),
                                          self._p(u_row0) if u_row0 is not None else None, self._p(y)))
        return y

    def kx(self, row0, r):
        z = self.empty(r.shape[0], self.Nx)
        _lib.check(self.lib.st_rows_KX(self.h, row0, r.shape[0], self._p(r), self._p(z)))
        return z

    def wavelet_cols(self, synthesize, cols):
        out = self.empty(cols.shape[0], cols.shape[1])
        _lib.check(self.lib.st_wavelet_cols(self.h, 1 if synthesize else 0, cols.shape[1], self._p(cols),
                                            self._p(out)))
        return out

    def dot(self, a, b):
        res = ctypes.c_double()
        _lib.check(self.lib.st_vec_dot(self.h, a.numel(), self._p(a), self._p(b), ctypes.byref(res)))
        return res.value

    def axpby(self, alpha, x, beta, y):
        _lib.check(self.lib.st_vec_axpby(self.h, x.numel(), alpha, self._p(x), beta, self._p(y)))

    def sync(self):
        self.solver.stream.synchronize()

    def close(self):
        self.solver.close()


# ----------------------------------------------------------------------------------------------
# the compiled sharded solve: st_sharded_solve runs the right-hand side, the PCG (scalars, stop
# test, updates) and the synthesis; Python only lends it the communicator
# ----------------------------------------------------------------------------------------------
class _DeviceArray:
    """A device buffer of the library seen as a torch tensor (no copy)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _device_tensor(ptr, n):
    import torch
    return torch.as_tensor(_DeviceArray(ptr, n), device="cuda")


def make_st_comm(comm):
    """st_comm callbacks over a communicator with exchange(sends, recvs) and allreduce_sum(x);
    returns (struct, keep-alive objects)."""
    P = comm.size if comm is not None else 0

    def allreduce(_ctx, v, n):
        try:
            for i in range(n):
                v[i] = comm.allreduce_sum(v[i])
            return 0
        except Exception:
            return 1

    def exchange(_ctx, send, nsend, recv, nrecv):
        try:
            sends = {s: _device_tensor(send[s], nsend[s]) for s in range(P) if nsend[s] > 0}
            recvs = {s: _device_tensor(recv[s], nrecv[s]) for s in range(P) if nrecv[s] > 0}
            comm.exchange(sends, recvs)
            return 0
        except Exception:
            return 1

    a, e = _lib.ALLREDUCE_FN(allreduce), _lib.EXCHANGE_FN(exchange)
    return _lib.StComm(None, a, e), (a, e)


def sharded_solve(backend, comm, g_rows, u0):
    """The rank's rows of u for its rows of g and u0 (N_x, read by the rank owning row 0), with
    the time axis split over the ranks of `comm` (st_sharded_solve; `backend` a CudaBackend whose
    handle carries the tolerance).  Returns (u rows, iterations, relres)."""
    import torch
    check_partition(backend.J, comm.size)
    lo, hi = row_range(backend.J, comm.size, comm.rank)
    if tuple(g_rows.shape) != (hi - lo, backend.Nx) or not g_rows.is_cuda or not u0.is_cuda:
        raise ValueError("g_rows must be this rank's (rows, N_x) CUDA tensor and u0 a CUDA tensor")
    u = torch.empty_like(g_rows)
    st_comm, keep = make_st_comm(comm)
    its, rr = ctypes.c_int(), ctypes.c_double()
    torch.cuda.synchronize()
    st = backend.lib.st_sharded_solve(backend.h, ctypes.byref(st_comm), comm.rank, comm.size,
                                      ctypes.c_void_p(g_rows.data_ptr()), ctypes.c_void_p(u0.data_ptr()),
                                      ctypes.c_void_p(u.data_ptr()), ctypes.byref(its), ctypes.byref(rr))
    del keep
    if st not in (_lib.ST_OK,):
        _lib.check(st)
    return u, its.value, rr.value


# ----------------------------------------------------------------------------------------------
# the sharded solver's schedule in Python (the CPU backend of the gloo tests drives it)
# ----------------------------------------------------------------------------------------------
class TimeShardedSolver:
    """PCG on S_hat w = f_hat (Sec. 3.4) with the time rows of every vector split over the ranks
    of `comm`; `backend` computes on the local rows (or columns)."""

    def __init__(self, J, comm, backend):
        check_partition(J, comm.size)
        self.J, self.comm, self.be = J, comm, backend
        self.P, self.rank = comm.size, comm.rank
        self.Nt, self.Nx = backend.Nt, backend.Nx
        self.lo, self.hi = row_range(J, self.P, self.rank)
        self.nrows = self.hi - self.lo
        self.rows = [row_range(J, self.P, r) for r in range(self.P)]
        self.cols = [col_range(self.Nx, self.P, r) for r in range(self.P)]

    # -- exchanges -----------------------------------------------------------------------------
    def rows_to_cols(self, X):
        """(nrows, N_x) of this rank -> (N_t, ncols) of this rank's columns."""
        c0, c1 = self.cols[self.rank]
        out = self.be.empty(self.Nt, c1 - c0)
        sends = {s: X[:, a:b].contiguous() for s, (a, b) in enumerate(self.cols)}
        recvs = {s: self.be.empty(hi - lo, c1 - c0) for s, (lo, hi) in enumerate(self.rows)}
        self._sync()
        self.comm.exchange(sends, recvs)
        for s, (lo, hi) in enumerate(self.rows):
            out[lo:hi] = recvs[s]
        return out

    def cols_to_rows(self, C):
        """(N_t, ncols) of this rank's columns -> (nrows, N_x) of this rank's rows."""
        out = self.be.empty(self.nrows, self.Nx)
        sends = {s: C[lo:hi].contiguous() for s, (lo, hi) in enumerate(self.rows)}
        recvs = {s: self.be.empty(self.nrows, b - a) for s, (a, b) in enumerate(self.cols)}
        self._sync()
        self.comm.exchange(sends, recvs)
        for s, (a, b) in enumerate(self.cols):
            out[:, a:b] = recvs[s]
        return out

    def halo(self, U):
        """U's rows with one neighbour row each side (zeros beyond the time axis)."""
        H = self.be.zeros(self.nrows + 2, self.Nx)
        H[1:-1] = U
        sends, recvs = {}, {}
        if self.rank > 0:
            sends[self.rank - 1] = U[:1].contiguous()
            recvs[self.rank - 1] = self.be.empty(1, self.Nx)
        if self.rank < self.P - 1:
            sends[self.rank + 1] = U[-1:].contiguous()
            recvs[self.rank + 1] = self.be.empty(1, self.Nx)
        self._sync()
        self.comm.exchange(sends, recvs)
        if self.rank > 0:
            H[0] = recvs[self.rank - 1][0]
        if self.rank < self.P - 1:
            H[-1] = recvs[self.rank + 1][0]
        return H

    def _sync(self):
        if hasattr(self.be, "sync"):
            self.be.sync()

    # -- operators (every argument and result: this rank's rows) ------------------------------
    def synthesize(self, w):
        return self.cols_to_rows(self.be.wavelet_cols(True, self.rows_to_cols(w)))

    def analyze(self, u):
        return self.cols_to_rows(self.be.wavelet_cols(False, self.rows_to_cols(u)))

    def apply_S_nodal(self, u):
        H = self.halo(u)
        return self.be.nodal(0, self.lo, H, H[1] if self.lo == 0 else None)

    def apply_Shat(self, w):
        return self.analyze(self.apply_S_nodal(self.synthesize(w)))

    def apply_KX(self, r):
        return self.be.kx(self.lo, r)

    def rhs(self, g, u0):
        """f_hat rows from the nodal g rows and u0 (N_x; read by the rank that owns row 0)."""
        H = self.halo(g)
        return self.analyze(self.be.nodal(1, self.lo, H, u0 if self.lo == 0 else None))

    def dot(self, a, b):
        return self.comm.allreduce_sum(self.be.dot(a, b))

    # -- PCG (Sec. 3.4, Eq. 3.3), stopping as the single-GPU solver ------------------------------
    def pcg(self, fhat, tol=1e-10, tol_mode=0, maxit=200):
        """Returns (w rows, iterations, sqrt(r^T K_X r / r_0^T K_X r_0))."""
        w = self.be.zeros(self.nrows, self.Nx)
        r = fhat.clone()
        z = self.apply_KX(r)
        rho = self.dot(r, z)
        rho0 = rho
        p = z.clone()
        rel = 0.0
        if rho0 == 0.0 or (tol_mode == 1 and math.sqrt(rho0) <= tol):
            return w, 0, rel
        for it in range(1, maxit + 1):
            q = self.apply_Shat(p)
            pq = self.dot(p, q)
            if not (pq > 0.0) or not math.isfinite(pq):
                raise _lib.STError(_lib.ST_ERR_BREAKDOWN, "time-sharded PCG: p^T S_hat p <= 0")
            alpha = rho / pq
            self.be.axpby(alpha, p, 1.0, w)
            self.be.axpby(-alpha, q, 1.0, r)
            z = self.apply_KX(r)
            rho_new = self.dot(r, z)
            rel = math.sqrt(rho_new / rho0)
            if (tol_mode == 1 and math.sqrt(rho_new) <= tol) or (tol_mode == 0 and rel <= tol):
                return w, it, rel
            self.be.axpby(1.0, z, rho_new / rho, p)
            rho = rho_new
        return w, maxit, rel

    def solve(self, g, u0, tol=1e-10, tol_mode=0, maxit=200):
        """u rows (nodal) of the solution for g rows and u0; returns (u, iterations, relres)."""
        w, its, rel = self.pcg(self.rhs(g, u0), tol, tol_mode, maxit)
        return self.synthesize(w), its, rel
