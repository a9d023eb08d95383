// molt_wave_step_noalloc: one wave time step that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a fixed device-
// memory budget, or inside a framework whose caching allocator owns all of the
// device's memory, and code on latency-critical paths where a first-use
// allocation (and the synchronisation it implies) is not acceptable.  They can
// still advance a small 1-, 2- or 3-D wave problem with this entry point.  Its
// scratch -- the FP32 copy of u^n the sweeps read, the FP32 axis accumulator
// and the status word -- lives in the file-scope device array below, which
// every GPU that loads the library holds until the process exits.  The caller
// passes u^n, u^{n-1} and the output u^{n+1}.  The sweep kernels are the ones
// molt_step runs (plain one-tile-per-CTA variant).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "coeffs.h"
#include "line_constants.h"
#include "molt.h"
#include "sweep_launch.h"

using namespace molt;

namespace {

constexpr long long kNoAllocMaxPoints = 1LL << 20;     // 1,048,576 grid points
constexpr size_t kStatusBytes = 256;
constexpr size_t kScratchBytes = kStatusBytes + 2 * 4 * size_t(kNoAllocMaxPoints);  // 8 MiB + 256 B
constexpr int kMaxDevices = 64;

// Shared by every call on a device: status word, FP32 accumulator, FP32 copy.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host-side device address of g_noalloc_scratch, looked up once per device
// and CUDA context (the symbol's name in host code is only a stand-in, never
// a device address).  The context is part of the key: after cudaDeviceReset,
// or whenever the primary context is destroyed and created again, the module
// loads again and the array may sit at another address, so a new context
// means a new lookup.  The mutex orders first calls from several host threads.
struct ScratchAddr {
  CUcontext ctx = nullptr;
  void* ptr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// cuCtxGetCurrent through the runtime's driver entry point (the library does
// not link the driver library itself).
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Device address of the scratch array for the current device and context;
// nullptr on failure.
void* scratch_address(int dev) {
  CtxGetCurrentFn get = ctx_get_current();
  CUcontext cur = nullptr;
  if (!get || get(&cur) != CUDA_SUCCESS) return nullptr;
  if (!cur) {
    // no context current on this thread yet: the runtime's first call (the
    // lookup itself) makes the device's primary context current
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return nullptr;
    }
    if (get(&cur) != CUDA_SUCCESS || !cur) return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ScratchAddr& e = g_scratch_addr[dev];
  if (e.ctx != cur || !e.ptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return nullptr;
    }
    e.ctx = cur;
    e.ptr = p;
  }
  return e.ptr;
}

__global__ void noalloc_copy_kernel(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = d2f(in[i]);
}

int phys_len(int e) {
  const int ee = e + kG;
  return ee + (ee >> 4);
}

// Kernel arguments of the sum_{p<=P} D_0^p sweep along `ax` (same tile rules
// as molt_step's planner).  Returns false if the line does not fit.
bool plan(const molt_desc& d, int ax, double alpha, int* status, SweepArgs* a, int* grid, int* block,
          size_t* smem) {
  std::memset(a, 0, sizeof(*a));
  const long long nx = d.n[0], ny = d.ndim > 1 ? d.n[1] : 1, nz = d.ndim > 2 ? d.n[2] : 1;
  LineGeom& g = a->g;
  if (ax == 0) {
    g.n = int(nx); g.nlines = ny * nz; g.nlo = ny; g.s_lo = nx; g.s_hi = nx * ny; g.stride = 1;
  } else if (ax == 1) {
    g.n = int(ny); g.nlines = nx * nz; g.nlo = nx; g.s_lo = 1; g.s_hi = nx * ny; g.stride = nx;
  } else {
    g.n = int(nz); g.nlines = nx * ny; g.nlo = nx; g.s_lo = 1; g.s_hi = nx; g.stride = nx * ny;
  }
  const int n = g.n;
  a->bc = d.bc[ax];
  a->mode = MODE_0;
  a->P = d.P;
  a->contiguous = g.stride == 1;
  a->alpha = alpha;
  const int N = a->bc == MOLT_BC_PERIODIC ? n : n - 1;
  const double h = (d.hi[ax] - d.lo[ax]) / double(N);
  const double nu = alpha * h;
  QuadTable qt;
  if (!(nu > 0) || !std::isfinite(nu) || !build_quadrature(d.quad_points, nu, &qt)) return false;
  set_line_constants(*a, qt, N, kE, true);   // FP32 sweeps
  const int nwl = (n + 32 * kE - 1) / (32 * kE);
  if (nwl > kMaxThreads / 32) return false;
  int W = 1;
  while (W * 2 <= (kMaxThreads / 32) / nwl) W *= 2;
  while (W > 1 && (long long)W / 2 >= g.nlines) W /= 2;
  int LS = phys_len(nwl * 32 * kE + 3) + 1;
  LS = (LS + 31) / 32 * 32 + (W < 32 ? 32 / W : 1);
  a->W = W;
  a->nwl = nwl;
  a->LS = LS;
  const size_t off = (size_t(4 * W) * 8 + size_t(W * nwl * 4) * 4 + 15) & ~size_t(15);
  *smem = off + size_t(W) * LS * 4;
  if (*smem > kSmemTileBudget) return false;
  *block = 32 * nwl * W;
  *grid = int((g.nlines + W - 1) / W);
  a->status = status;
  return true;
}

}  // namespace

extern "C" molt_status molt_wave_step_noalloc(const molt_desc* d, const double* u, const double* u_prev,
                                              double* u_next, int from_rest, void* cuda_stream) {
  if (!d || !u || !u_next || (!from_rest && !u_prev)) return MOLT_EINVAL;
  if (d->pde != MOLT_PDE_WAVE || d->prec != MOLT_PREC_F32_F64UPDATE || d->weights != MOLT_W_LINEAR)
    return MOLT_EUNSUPPORTED;
  if (d->ndim < 1 || d->ndim > 3 || d->P < 1 || d->P > 64 || !(d->dt > 0) || !(d->c > 0) || !(d->beta > 0))
    return MOLT_EINVAL;
  if (d->quad_points != 3 && d->quad_points != 5 && d->quad_points != 6) return MOLT_EINVAL;
  if (u_next == u) return MOLT_EINVAL;   // u_next may be u_prev, never u^n itself
  long long total = 1;
  for (int ax = 0; ax < d->ndim; ++ax) {
    if (d->n[ax] < 2 || d->n[ax] > 8192) return MOLT_EINVAL;
    if (d->bc[ax] != MOLT_BC_PERIODIC && d->bc[ax] != MOLT_BC_DIRICHLET) return MOLT_EINVAL;
    if (!(d->hi[ax] > d->lo[ax])) return MOLT_EINVAL;
    total *= d->n[ax];
  }
  if (total > kNoAllocMaxPoints) return MOLT_EINVAL;   // beyond the scratch array
  if ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(u_prev) | reinterpret_cast<uintptr_t>(u_next)) &
      15)
    return MOLT_EINVAL;

  // Set-up, once per device and context: the device address of the scratch array.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MOLT_ECUDA;
  unsigned char* base = static_cast<unsigned char*>(scratch_address(dev));
  if (!base) return MOLT_ECUDA;
  int* status = reinterpret_cast<int*>(base);
  float* acc = reinterpret_cast<float*>(base + kStatusBytes);
  float* copy = acc + kNoAllocMaxPoints;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  // the status word keeps the previous call's value: clear it
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return MOLT_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (total + 255) / 256;
  if (blocks > 8LL * (sms > 0 ? sms : 1)) blocks = 8LL * (sms > 0 ? sms : 1);
  noalloc_copy_kernel<<<int(blocks), 256, 0, s>>>(u, copy, total);
  if (cudaGetLastError() != cudaSuccess) return MOLT_ECUDA;

  const double alpha = d->beta / (d->c * d->dt);
  for (int ax = 0; ax < d->ndim; ++ax) {
    SweepArgs a;
    int grid = 0, block = 0;
    size_t smem = 0;
    if (!plan(*d, ax, alpha, status, &a, &grid, &block, &smem)) return MOLT_EUNSUPPORTED;
    a.in = copy;
    a.acc = acc;
    cudaError_t e;
    if (ax + 1 < d->ndim) {
      e = ax == 0 ? launch_sweep<float, float, double, false, EPI_ACC_SET>(a, nullptr, grid, block, smem, s)
                  : launch_sweep<float, float, double, false, EPI_ACC_ADD>(a, nullptr, grid, block, smem, s);
    } else {
      if (d->ndim == 1) a.acc = nullptr;
      a.un = u;
      a.us = u_prev;
      a.dst = u_next;
      a.coefS = -d->beta * d->beta;
      a.from_rest = from_rest ? 1 : 0;
      e = launch_sweep<float, float, double, false, EPI_WAVE_FINAL>(a, nullptr, grid, block, smem, s);
    }
    if (e != cudaSuccess) return MOLT_ECUDA;
  }
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MOLT_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MOLT_ECUDA;
  if (h_status & ST_NONFINITE) return MOLT_ENONFINITE;
  return MOLT_OK;
}
