// Nested iteration (Sec. 4.4, after Hackbusch Ch. 5): solve on the meshes (K - m, J - m),
// m = levels-1 .. 0, each PCG started from the previous level's solution and stopped at the
// absolute K_X-norm tolerance eps 2^(rate m) (Eq. 3.3), so that the algebraic error follows the
// discretisation error from level to level.
//
// Both transfers are exact embeddings.  Nodal data move to a coarser mesh by injection (coarse
// time node t is fine node 2t, coarse grid node (i, j) is fine grid node (2i, 2j)).  A solution
// in wavelet coordinates moves to the next finer mesh unchanged in time: in the in-place row
// order, coarse row i is fine row 2i (the coarse wavelets are the first fine ones, Eq. 3.1), the
// new level's details (odd rows) are 0; in space each row is written in the fine P1 basis
// (the multigrid's nested prolongation).
#include <cmath>
#include <cstring>
#include <string>

#include "st_internal.cuh"

namespace st {
namespace {

// coarse (b, t, iy, ix) = fine (b, tstep t, 2 iy + 1, 2 ix + 1); u0 uses ntc = ntf = 1, tstep 0
__global__ void __launch_bounds__(256) k_inject(double* __restrict__ c, const double* __restrict__ f, int nc, int nf,
                                                int64_t ntc, int64_t ntf, int tstep) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nc * nc) return;
  const int iy = p / nc, ix = p - iy * nc;
  const int64_t t = blockIdx.y, b = blockIdx.z;
  c[(b * ntc + t) * nc * nc + p] = f[(b * ntf + t * tstep) * nf * nf + (int64_t)(2 * iy + 1) * nf + 2 * ix + 1];
}

// fine in-place row i: the P1 prolongation of coarse row i / 2 for even i, 0 for odd i
__global__ void __launch_bounds__(256) k_prolong_w(double* __restrict__ wf, const double* __restrict__ wc, int nf,
                                                   int nc, int64_t ntf, int64_t ntc, int lshape) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nf * nf) return;
  const int iy = p / nf, ix = p - iy * nf;
  const int64_t i = blockIdx.y, b = blockIdx.z;
  double v = 0.0;
  if (!(i & 1) && !outside_domain(ix, iy, nf, lshape))
    v = prolong_value<double>(wc + (b * ntc + i / 2) * nc * nc, nc, ix + 1, iy + 1);
  wf[(b * ntf + i) * nf * nf + p] = v;
}

// the cube: coarse (b, t, z, y, x) = fine (b, tstep t, 2z + 1, 2y + 1, 2x + 1)
__global__ void __launch_bounds__(256) k_inject3(double* __restrict__ c, const double* __restrict__ f, int nc, int nf,
                                                 int64_t ntc, int64_t ntf, int tstep) {
  const int64_t Nc = (int64_t)nc * nc * nc;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= Nc) return;
  const int ix = (int)(p % nc), iy = (int)((p / nc) % nc), iz = (int)(p / ((int64_t)nc * nc));
  const int64_t t = blockIdx.y, b = blockIdx.z;
  const int64_t Nf = (int64_t)nf * nf * nf;
  c[(b * ntc + t) * Nc + p] =
      f[(b * ntf + t * tstep) * Nf + ((int64_t)(2 * iz + 1) * nf + (2 * iy + 1)) * nf + 2 * ix + 1];
}

__global__ void __launch_bounds__(256) k_prolong_w3(double* __restrict__ wf, const double* __restrict__ wc, int nf,
                                                    int nc, int64_t ntf, int64_t ntc) {
  const int64_t Nf = (int64_t)nf * nf * nf;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= Nf) return;
  const int ix = (int)(p % nf), iy = (int)((p / nf) % nf), iz = (int)(p / ((int64_t)nf * nf));
  const int64_t i = blockIdx.y, b = blockIdx.z;
  double v = 0.0;
  if (!(i & 1)) v = prolong_value3<double>(wc + (b * ntc + i / 2) * nc * nc * nc, nc, ix + 1, iy + 1, iz + 1);
  wf[(b * ntf + i) * Nf + p] = v;
}

cudaError_t inject(const st_handle_s* fine, const st_handle_s* coarse, const double* f, double* c, bool time) {
  const int nc = coarse->n, nf = fine->n;
  if (fine->domain == 2) {
    const int64_t ntc = time ? coarse->Nt : 1, ntf = time ? fine->Nt : 1;
    dim3 grid((unsigned)((coarse->Nx + 255) / 256), (unsigned)ntc, fine->B);
    k_inject3<<<grid, 256, 0, fine->stream>>>(c, f, nc, nf, ntc, ntf, time ? 2 : 0);
    count_launch(fine);
    return cudaGetLastError();
  }
  const int64_t ntc = time ? coarse->Nt : 1, ntf = time ? fine->Nt : 1;
  dim3 grid((nc * nc + 255) / 256, (unsigned)ntc, fine->B);
  k_inject<<<grid, 256, 0, fine->stream>>>(c, f, nc, nf, ntc, ntf, time ? 2 : 0);
  count_launch(fine);
  return cudaGetLastError();
}

cudaError_t prolong_w(const st_handle_s* coarse, const st_handle_s* fine, const double* wc, double* wf) {
  const int nf = fine->n;
  if (fine->domain == 2) {
    dim3 grid((unsigned)((fine->Nx + 255) / 256), (unsigned)fine->Nt, fine->B);
    k_prolong_w3<<<grid, 256, 0, fine->stream>>>(wf, wc, nf, coarse->n, fine->Nt, coarse->Nt);
    count_launch(fine);
    return cudaGetLastError();
  }
  dim3 grid((nf * nf + 255) / 256, (unsigned)fine->Nt, fine->B);
  k_prolong_w<<<grid, 256, 0, fine->stream>>>(wf, wc, nf, coarse->n, fine->Nt, coarse->Nt, fine->domain);
  count_launch(fine);
  return cudaGetLastError();
}

}  // namespace
}  // namespace st

using namespace st;

extern "C" {

st_status st_nested_solve(st_handle h, int levels, double eps, double rate, const double* g, const double* u0,
                          double* w, int* iters_per_level) {
  if (!h || !g || !u0 || !w) {
    set_error("st_nested_solve: null handle or pointer");
    return ST_ERR_ARG;
  }
  const int kmin = h->domain == 1 ? 2 : 1;
  if (levels < 1 || levels > 16 || h->K - levels + 1 < kmin || h->J - levels + 1 < 1) {
    set_error("st_nested_solve: levels must be in 1..16 with the coarsest mesh (K - levels + 1, J - levels + 1) "
              "at least (" + std::to_string(kmin) + ", 1)");
    return ST_ERR_ARG;
  }
  if (!(eps > 0.0) || !std::isfinite(eps) || !std::isfinite(rate)) {
    set_error("st_nested_solve: eps must be positive and rate finite");
    return ST_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail("cudaSetDevice", e);
  // coarser handles, created once with the fine handle's settings and Gauss-Seidel choices
  for (int m = 1; m < levels; ++m) {
    if (h->nest[m]) continue;
    st_status s = st_setup_batch(&h->nest[m], h->domain, h->K - m, h->J - m, h->B, &h->cfg, h->stream);
    if (s != ST_OK) return s;
    std::memcpy(h->nest[m]->gs_kind, h->gs_kind, sizeof(h->gs_kind));
    std::memcpy(h->nest[m]->gs_seg, h->gs_seg, sizeof(h->gs_seg));
  }
  // data of every level by injection from the next finer one
  for (int m = 1; m < levels; ++m) {
    st_handle_s* f = m == 1 ? h : h->nest[m - 1];
    st_handle_s* c = h->nest[m];
    if ((e = inject(f, c, m == 1 ? g : f->g, c->g, true)) != cudaSuccess) return cuda_fail("injection of g", e);
    if ((e = inject(f, c, m == 1 ? u0 : f->u0, c->u0, false)) != cudaSuccess) return cuda_fail("injection of u0", e);
  }
  st_status result = ST_OK;
  for (int m = levels - 1; m >= 0; --m) {
    st_handle_s* hm = m ? h->nest[m] : h;
    double* wm = m ? hm->w : w;
    st_status s = rhs_impl(hm, hm->B, m ? hm->g : g, m ? hm->u0 : u0, hm->fhat);
    if (s != ST_OK) return s;
    if (m < levels - 1) {
      st_handle_s* prev = h->nest[m + 1];
      if ((e = prolong_w(prev, hm, prev->w, wm)) != cudaSuccess) return cuda_fail("prolongation of w", e);
    }
    const double tol = hm->cfg.tol;
    const int tol_mode = hm->cfg.tol_mode;
    hm->cfg.tol = eps * std::exp2(rate * m);
    hm->cfg.tol_mode = 1;
    hm->use_guess = m < levels - 1;
    int its = 0;
    s = pcg_impl(hm, hm->fhat, wm, &its, nullptr);
    hm->use_guess = false;
    hm->cfg.tol = tol;
    hm->cfg.tol_mode = tol_mode;
    if (iters_per_level) iters_per_level[levels - 1 - m] = its;
    if (s != ST_OK && s != ST_ERR_MAXIT) return s;
    if (s == ST_ERR_MAXIT && result == ST_OK) result = s;
  }
  return result;
}

}  // extern "C"
