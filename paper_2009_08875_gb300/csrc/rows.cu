// Building blocks of a time-sharded solve (the paper distributes the time axis over processes,
// Sec. 5.2): every operator of a PCG iteration restricted to the time rows a rank owns, the
// wavelet transform of a block of columns, and the binary64 vector operations the iteration
// needs.  The handle (B = 1) provides the coefficient tables and the scratch; the caller's
// vectors hold only the rows (or columns) the call is about.
#include "st_internal.cuh"

using namespace st;

namespace {

st_status check_rows(st_handle h, int64_t row0, int64_t nrows, const char* who) {
  if (!h) {
    set_error(std::string(who) + ": null handle");
    return ST_ERR_ARG;
  }
  if (h->B != 1 || row0 < 0 || nrows < 1 || row0 + nrows > h->Nt) {
    set_error(std::string(who) + ": needs a single-problem handle and rows 0 <= row0 < row0 + nrows <= N_t");
    return ST_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail("cudaSetDevice", e);
  return ST_OK;
}

}  // namespace

extern "C" {

st_status st_rows_nodal(st_handle h, int mode, int64_t row0, int64_t nrows, const double* u_halo,
                        const double* u_row0, double* y) {
  st_status s = check_rows(h, row0, nrows, "st_rows_nodal");
  if (s != ST_OK) return s;
  if (!u_halo || !y || (mode != 0 && mode != 1)) {
    set_error("st_rows_nodal: null pointer or mode not 0 / 1");
    return ST_ERR_ARG;
  }
  cudaError_t e = launch_timemix_rows(h, mode, (int)row0, (int)nrows, u_halo, h->Y);
  if (e == cudaSuccess) e = mg_apply<double>(h, (int)(2 * nrows), 0, h->Y, h->X);
  if (e == cudaSuccess) e = launch_epilogue_rows(h, (int)row0, (int)nrows, h->X, row0 == 0 ? u_row0 : nullptr, y);
  if (e != cudaSuccess) return cuda_fail("st_rows_nodal", e);
  return ST_OK;
}

st_status st_rows_KX(st_handle h, int64_t row0, int64_t nrows, const double* r, double* z) {
  st_status s = check_rows(h, row0, nrows, "st_rows_KX");
  if (s != ST_OK) return s;
  if (!r || !z) {
    set_error("st_rows_KX: null pointer");
    return ST_ERR_ARG;
  }
  const int cls = (int)(-1 - row0);  // per-slice K_l of wavelet row row0 + slice
  cudaError_t e = mg_apply<double>(h, (int)nrows, cls, r, h->X);
  if (e == cudaSuccess) e = launch_apply_A<double>(h, (int)nrows, h->X, h->Y);
  if (e == cudaSuccess) e = mg_apply<double>(h, (int)nrows, cls, h->Y, z);
  if (e != cudaSuccess) return cuda_fail("st_rows_KX", e);
  return ST_OK;
}

st_status st_wavelet_cols(st_handle h, int synthesize, int64_t ncols, const double* in, double* out) {
  if (!h || !in || !out || ncols < 1 || ncols > h->Nx || h->B != 1) {
    set_error("st_wavelet_cols: null pointer, single-problem handle needed, or ncols not in 1..N_x");
    return ST_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e == cudaSuccess) e = wavelet_cols(h, synthesize ? 1 : 0, ncols, in, out);
  if (e != cudaSuccess) return cuda_fail("st_wavelet_cols", e);
  return ST_OK;
}

st_status st_vec_dot(st_handle h, int64_t n, const double* a, const double* b, double* result) {
  if (!h || !a || !b || !result || n < 1) {
    set_error("st_vec_dot: null pointer or n < 1");
    return ST_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e == cudaSuccess) e = launch_dot<double, double>(h, 0, 1, a, b, n, SC_OUTER, DOT_STORE);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(result, h->scal + SC_OUTER, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail("st_vec_dot", e);
  return ST_OK;
}

st_status st_vec_axpby(st_handle h, int64_t n, double alpha, const double* x, double beta, double* y) {
  if (!h || !x || !y || n < 1) {
    set_error("st_vec_axpby: null pointer or n < 1");
    return ST_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e == cudaSuccess) e = launch_axpby(h, y, x, alpha, beta, n);
  if (e != cudaSuccess) return cuda_fail("st_vec_axpby", e);
  return ST_OK;
}

}  // extern "C"
