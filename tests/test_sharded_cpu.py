"""The time-sharded PCG schedule (paper_2009_08875_gb300.sharded) on CPU ranks with gloo.

The ranks run the sharded solver's exchanges (neighbour rows for the time mix, rows <-> columns
for the wavelet transforms, sums of partial inner products) through torch.distributed with the
gloo backend, and a CPU backend that evaluates each rank's local operators with the oracle (the
operators are local in the sense the schedule needs: S's nodal rows depend on the neighbour rows
only, K_X is block diagonal in the wavelet rows, W acts on each column separately).  Every rank's
rows of f_hat, of S_hat applied to a random vector, and of the PCG solution must match the
unsharded oracle, with the same iteration count.  World sizes 2 and 4.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

K, J = 3, 3


class OracleRowsBackend:
    """Local operators of one rank evaluated with the oracle on CPU tensors."""

    def __init__(self, prob):
        self.p = prob
        self.Nt, self.Nx, self.J = prob.Nt, prob.Nx, prob.J

    def empty(self, rows, cols):
        return torch.empty((rows, cols), dtype=torch.float64)

    def zeros(self, rows, cols):
        return torch.zeros((rows, cols), dtype=torch.float64)

    def _full(self, row0, halo):
        F = np.zeros((self.Nt, self.Nx))
        a, b = row0 - 1, row0 - 1 + halo.shape[0]
        lo, hi = max(a, 0), min(b, self.Nt)
        F[lo:hi] = halo.numpy()[lo - a:hi - a]
        return F

    def nodal(self, mode, row0, u_halo, u_row0):
        nrows = u_halo.shape[0] - 2
        F = self._full(row0, u_halo)
        if mode == 0:
            Y = self.p.apply_S_route2(F)
        else:
            u0 = u_row0.numpy() if u_row0 is not None else np.zeros(self.Nx)
            Y = self.p.rhs(F, u0)
        return torch.from_numpy(np.ascontiguousarray(Y[row0:row0 + nrows]))

    def kx(self, row0, r):
        F = np.zeros((self.Nt, self.Nx))
        F[row0:row0 + r.shape[0]] = r.numpy()
        Z = self.p.to_inplace(self.p.apply_KX(self.p.from_inplace(F)))
        return torch.from_numpy(np.ascontiguousarray(Z[row0:row0 + r.shape[0]]))

    def wavelet_cols(self, synthesize, cols):
        C = cols.numpy()
        out = self.p.synth(self.p.from_inplace(C)) if synthesize else self.p.to_inplace(self.p.analysis(C))
        return torch.from_numpy(np.ascontiguousarray(out))

    def dot(self, a, b):
        return float(torch.sum(a * b))

    def axpby(self, alpha, x, beta, y):
        y.mul_(beta).add_(x, alpha=alpha)


def _worker(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import schur
        from paper_2009_08875_gb300 import inputs, sharded
        p = schur.Problem(K, J)
        comm = sharded.TorchComm()
        ts = sharded.TimeShardedSolver(J, comm, OracleRowsBackend(p))
        lo, hi = ts.lo, ts.hi
        g, u0, _ = inputs.manufactured(K, J)
        fhat_ref = p.to_inplace(p.rhs_hat(g, u0))
        fhat = ts.rhs(torch.from_numpy(np.ascontiguousarray(g[lo:hi])), torch.from_numpy(u0))
        err_f = float(np.abs(fhat.numpy() - fhat_ref[lo:hi]).max() / np.abs(fhat_ref).max())
        w = np.random.default_rng(5).standard_normal((p.Nt, p.Nx))
        q_ref = p.to_inplace(p.apply_Shat(p.from_inplace(w)))
        q = ts.apply_Shat(torch.from_numpy(np.ascontiguousarray(w[lo:hi])))
        err_q = float(np.abs(q.numpy() - q_ref[lo:hi]).max() / np.abs(q_ref).max())
        u, its, _ = ts.solve(torch.from_numpy(np.ascontiguousarray(g[lo:hi])), torch.from_numpy(u0), tol=1e-10)
        u_ref, _, info = schur.solve(p, g, u0, tol=1e-10)
        err_u = float(np.abs(u.numpy() - u_ref[lo:hi]).max() / np.abs(u_ref).max())
        out_q.put((rank, err_f, err_q, err_u, its, info["iters"]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 4])
def test_time_sharded_pcg_matches_oracle(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    results = [q.get(timeout=600) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, err_f, err_q, err_u, its, its_ref in results:
        assert err_f < 1e-13 and err_q < 1e-13, (rank, err_f, err_q)
        assert err_u < 1e-10 and its == its_ref, (rank, err_u, its, its_ref)


def test_partition_covers_the_time_axis_once():
    from paper_2009_08875_gb300 import sharded
    for Jt in (1, 3, 6):
        for P in (1, 2, 4, 8):
            if P > 2 ** Jt:
                with pytest.raises(ValueError):
                    sharded.check_partition(Jt, P)
                continue
            rows = [sharded.row_range(Jt, P, r) for r in range(P)]
            assert rows[0][0] == 0 and rows[-1][1] == 2 ** Jt + 1
            assert all(rows[i][1] == rows[i + 1][0] for i in range(P - 1))
            cols = [sharded.col_range(49, P, r) for r in range(P)]
            assert cols[0][0] == 0 and cols[-1][1] == 49
            assert all(cols[i][1] == cols[i + 1][0] for i in range(P - 1))
    with pytest.raises(ValueError):
        sharded.check_partition(4, 3)
