// st_apply_Kx_static: the K_x multigrid of st_apply_Kx for callers that cannot allocate device
// memory.  Such callers include processes in which another allocator owns the device memory
// budget (a framework's caching allocator or a serving runtime's arena, where a raw cudaMalloc
// can fail or fragment that pool) and latency-critical loops that forbid allocation after
// start-up because cudaMalloc/cudaFree may synchronise the device.  st_setup allocates a
// workspace, so this entry point needs no handle: its scratch is one file-scope device array.
//
// The multigrid work itself is the same code that st_apply_Kx runs (mg_apply on a handle
// description that lives on the host stack and points into the static array).
#include <cstring>
#include <mutex>
#include <string>

#include "st_internal.cuh"

namespace st {

// Maximum scratch: 32 MiB of doubles, held by every device that loads the library until exit.
constexpr size_t kStaticScratchDoubles = (size_t)4 << 20;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

cudaError_t mg_set_attributes();

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Resolves the device address of g_static_scratch on the current device (once per device).
// In host code the array's name is only a host-side stand-in, never a device address.
cudaError_t static_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    // the Gauss-Seidel kernels stage more than 48 KB of shared memory per block
    e = mg_set_attributes();
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Carves the buffers mg_apply needs for h->mg.max_slices slices at space level h->K out of
// the scratch starting at `base` (nullptr: only measure) and returns the doubles used: the
// coefficient table (classes 0..2, levels 0..K), the second fine iterate, the scaled fine
// right-hand side, and per coarse level two iterates and a right-hand side.  Every piece starts on a 256-byte boundary.
size_t carve_scratch(st_handle_s* h, double* base) {
  size_t used = 0;
  auto carve = [&](size_t count) {
    double* p = base ? base + used : nullptr;
    used += (count + 31) & ~(size_t)31;
    return p;
  };
  const size_t ns = (size_t)h->mg.max_slices;
  h->coef = reinterpret_cast<Coef<double>*>(carve((sizeof(Coef<double>) / sizeof(double)) * 3 * (h->K + 1)));
  h->Xalt = carve((size_t)h->Nx * ns);
  h->Bs = carve((size_t)h->Nx * ns);
  for (int k = 1; k <= h->K; ++k) {
    const size_t nk = (size_t)((1 << k) - 1) * ((1 << k) - 1) * ns;
    if (k < h->K) {
      h->mg.xc[k] = carve(nk);
      h->mg.xc2[k] = carve(nk);
      h->mg.bc[k] = carve(nk);
    }
  }
  return used;
}

}  // namespace

}  // namespace st

using namespace st;

extern "C" st_status st_apply_Kx_static(int space_level, int nslices, const double* b, double* x,
                                        void* cuda_stream) {
  // nslices is a grid dimension of the multigrid launches (65535 at most), as in st_setup
  if (space_level < 1 || space_level > 12 || nslices < 1 || nslices > 65535) {
    set_error("st_apply_Kx_static: space level must be in 1..12 and nslices in 1..65535");
    return ST_ERR_ARG;
  }
  if (!b || !x) {
    set_error("st_apply_Kx_static: null pointer");
    return ST_ERR_ARG;
  }
  // a handle description on the host stack whose buffers are carved out of the static array
  st_handle_s h;
  std::memset(&h, 0, sizeof(h));
  h.domain = 0;
  h.K = space_level;
  h.J = 1;  // coefficient classes 0..2; K_x uses class 0 only
  h.n = (1 << space_level) - 1;
  h.Nx = (int64_t)h.n * h.n;
  h.Nt = 3;
  st_default_config(&h.cfg);
  h.phys = Phys{1.0, 0.0, 1.0, 0.0};  // the heat equation's A_x
  h.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  h.mg.K = space_level;
  h.mg.kmin = 1;
  h.mg.max_slices = nslices;
  const size_t need = carve_scratch(&h, nullptr);
  if (need > kStaticScratchDoubles) {
    set_error("st_apply_Kx_static: " + std::to_string(nslices) + " slices at space level " +
              std::to_string(space_level) + " need " + std::to_string(need * sizeof(double)) +
              " bytes of scratch, more than the static maximum of " +
              std::to_string(kStaticScratchDoubles * sizeof(double)) + " bytes");
    return ST_ERR_ARG;
  }
  double* base = nullptr;
  cudaError_t e = static_scratch(&base);
  if (e != cudaSuccess) return cuda_fail("st_apply_Kx_static: device set-up (cudaGetSymbolAddress)", e);
  cudaGetDevice(&h.device);
  carve_scratch(&h, base);
  // Nothing in the scratch has to start at zero: every call rewrites the coefficient table, and
  // every multigrid buffer is written before it is read within the call (each coarse level, and
  // the finest level in the first cycle, start from x = 0 without reading the iterate buffer).
  e = launch_make_coef(h.coef, h.K, h.J, h.cfg.alpha, h.phys, 2, h.stream);
  if (e != cudaSuccess) return cuda_fail("st_apply_Kx_static: coefficient table", e);
  e = mg_apply(&h, nslices, 0, b, x);
  if (e != cudaSuccess) return cuda_fail("st_apply_Kx_static: multigrid", e);
  return ST_OK;
}
