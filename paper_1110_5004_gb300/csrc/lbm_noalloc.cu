// Allocation-free variant of the FP64 diagnostics reduction.
//
// Who needs it: a caller that cannot call cudaMalloc, because the host application already
// owns the device memory (a server that has reserved the whole budget for its own pools, or a
// solver loop that must not take the implicit device-wide synchronisation of a fresh
// allocation), can still reduce fields it holds.  It passes the four input fields and the
// output record; the per-row partial sums live in a fixed file-scope device array instead of
// memory the library would allocate.
//
// The array is shared by every call in the process on a given device and keeps the last
// call's contents.  Every partial a call reads is written earlier by the same call, so nothing
// has to start at zero; two calls whose kernels overlap on the GPU (different streams, no
// ordering between them) race on it and must not be issued.
#include <math.h>
#include <mutex>

#include "lbm_internal.h"

namespace lbm {

constexpr int NOALLOC_MAX_ROWS = 8192;
constexpr int NOALLOC_T = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

// 8192 rows x 12 partials + the 12-double result record: 768 KB held by every GPU that loads
// the library, until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_ROWS * DIAG_PARTIALS + 16];

__device__ __forceinline__ void na_tree_sum(double* sh, int t) {
  for (int s = NOALLOC_T / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
}
__device__ __forceinline__ void na_tree_max(double* sh, int t) {
  for (int s = NOALLOC_T / 2; s > 0; s >>= 1) {
    if (t < s) {
      const double a = sh[t], b = sh[t + s];
      sh[t] = (a >= b || a != a) ? a : b;
    }
    __syncthreads();
  }
}

// One block per row: the same partials, stride and tree as the simulation's diagnostics.
__global__ void __launch_bounds__(NOALLOC_T) k_noalloc_rows(double phs, int nx, int ny, const float* __restrict__ phi,
                                                            const float* __restrict__ ux, const float* __restrict__ uy,
                                                            const float* __restrict__ pp, double* __restrict__ part) {
  __shared__ double sh[DIAG_PARTIALS][NOALLOC_T];
  const int y = blockIdx.x, t = threadIdx.x;
  const long long o = (long long)y * nx;
  double acc[DIAG_PARTIALS] = {0};
  for (int x = t; x < nx; x += NOALLOC_T) {
    const double ph = phi[o + x], u = ux[o + x], v = uy[o + x], p = pp[o + x];
    double c = (ph + phs) / (2.0 * phs);
    c = c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c);
    acc[0] += ph;
    acc[1] += c;
    acc[2] += c * x;
    acc[3] += c * y;
    acc[4] += c * u;
    acc[5] += c * v;
    const double um = sqrt(u * u + v * v);
    if (!(um <= acc[6])) acc[6] = um;
    if (ph > 0.9 * phs) { acc[7] += p; acc[8] += 1.0; }
    if (ph < -0.9 * phs) { acc[9] += p; acc[10] += 1.0; }
  }
  for (int k = 0; k < 11; ++k) sh[k][t] = acc[k];
  __syncthreads();
  for (int k = 0; k < 11; ++k) {
    if (k == 6) na_tree_max(sh[k], t); else na_tree_sum(sh[k], t);
  }
  if (t < 11) part[(long long)y * DIAG_PARTIALS + t] = sh[t][0];
  if (t == 11) part[(long long)y * DIAG_PARTIALS + 11] = 0.0;
}

__global__ void __launch_bounds__(NOALLOC_T) k_noalloc_final(int ny, const double* __restrict__ part,
                                                             double* __restrict__ out, long long step) {
  __shared__ double sh[DIAG_PARTIALS][NOALLOC_T];
  const int t = threadIdx.x;
  double acc[DIAG_PARTIALS] = {0};
  for (int y = t; y < ny; y += NOALLOC_T) {
    const double* r = part + (long long)y * DIAG_PARTIALS;
    for (int k = 0; k < 11; ++k) {
      if (k == 6) {
        if (!(r[6] <= acc[6])) acc[6] = r[6];
      } else {
        acc[k] += r[k];
      }
    }
    if (!(r[1] <= acc[11])) acc[11] = r[1];
  }
  for (int k = 0; k < DIAG_PARTIALS; ++k) sh[k][t] = acc[k];
  __syncthreads();
  for (int k = 0; k < DIAG_PARTIALS; ++k) {
    if (k == 6 || k == 11) na_tree_max(sh[k], t); else na_tree_sum(sh[k], t);
  }
  if (t == 0) {
    lbm_diag d;
    d.step = step;
    d.sum_phi = sh[0][0];
    d.liquid_area = sh[1][0];
    const double sc = sh[1][0];
    d.centroid_x = sc > 0 ? sh[2][0] / sc : 0.0;
    d.centroid_y = sc > 0 ? sh[3][0] / sc : 0.0;
    d.vel_x = sc > 0 ? sh[4][0] / sc : 0.0;
    d.vel_y = sc > 0 ? sh[5][0] / sc : 0.0;
    d.spread_radius = 0.5 * sh[11][0];
    d.max_u = sh[6][0];
    d.p_liquid = sh[8][0] > 0 ? sh[7][0] / sh[8][0] : 0.0;
    d.p_gas = sh[10][0] > 0 ? sh[9][0] / sh[10][0] : 0.0;
    d.finite = isfinite(d.sum_phi) && isfinite(d.max_u);
    d.pad = 0;
    *reinterpret_cast<lbm_diag*>(out) = d;
  }
}

// Device address of the scratch array, looked up once per device with that device current.
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

static int noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_diagnostics_fields_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    set_error("lbm_diagnostics_fields_noalloc: device %d beyond the %d supported", dev, NOALLOC_MAX_DEVICES);
    return LBM_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "lbm_diagnostics_fields_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return LBM_OK;
}

// Memory the current device's kernels can address: managed memory, or device memory of this
// device (a field on another GPU would need peer access the library does not set up).
static bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

}  // namespace lbm

using namespace lbm;

extern "C" int lbm_diagnostics_fields_noalloc(const float* phi, const float* ux, const float* uy, const float* p,
                                              int nx, int ny, double phi_star, long long step, void* cuda_stream,
                                              lbm_diag* out) {
  if (!phi || !ux || !uy || !p || !out) return set_error("fields and out are required"), LBM_ERR_INVALID_ARG;
  if (nx < 1 || ny < 1) return set_error("grid %dx%d is empty", nx, ny), LBM_ERR_INVALID_ARG;
  if (ny > NOALLOC_MAX_ROWS) {
    set_error("lbm_diagnostics_fields_noalloc: ny = %d exceeds the fixed scratch of %d rows", ny, NOALLOC_MAX_ROWS);
    return LBM_ERR_INVALID_ARG;
  }
  if (!(phi_star > 0)) return set_error("phi_star must be positive"), LBM_ERR_INVALID_ARG;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_diagnostics_fields_noalloc: cudaGetDevice");
  if (!on_device(phi, dev) || !on_device(ux, dev) || !on_device(uy, dev) || !on_device(p, dev))
    return set_error("lbm_diagnostics_fields_noalloc: fields must be memory of the current device"),
           LBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const bool host_out = !on_device(out, dev);
  if (host_out) {
    // a host record needs a stream synchronisation, which a stream under capture refuses
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cs)) != cudaSuccess)
      return cuda_fail(e, "lbm_diagnostics_fields_noalloc: cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone)
      return set_error("lbm_diagnostics_fields_noalloc: a host out cannot be filled on a capturing stream; "
                       "pass a device out"), LBM_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  double* record = scratch + (long long)NOALLOC_MAX_ROWS * DIAG_PARTIALS;
  k_noalloc_rows<<<ny, NOALLOC_T, 0, st>>>(phi_star, nx, ny, phi, ux, uy, p, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "lbm_diagnostics_fields_noalloc: row kernel");
  k_noalloc_final<<<1, NOALLOC_T, 0, st>>>(ny, scratch, record, step);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "lbm_diagnostics_fields_noalloc: final kernel");
  e = cudaMemcpyAsync(out, record, sizeof(lbm_diag), host_out ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && host_out) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_diagnostics_fields_noalloc: result copy");
  if (host_out && !out->finite) {
    set_error("fields are not finite (step %lld)", step);
    return LBM_ERR_DIVERGED;
  }
  return LBM_OK;
}
