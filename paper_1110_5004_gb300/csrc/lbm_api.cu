// Host runtime and C ABI of liblbm: simulation objects, parameter checks, field transfer,
// step launches and diagnostics.  See include/lbm.h for the contract of every entry point.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <initializer_list>
#include <new>
#include <string>

#include "lbm_internal.h"

namespace lbm {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

Phys make_phys(const lbm_params& p) {
  Phys P{};
  const double cs2 = 1.0 / 3.0;
  P.four_beta = (float)(4.0 * p.beta);
  P.kappa = (float)p.kappa;
  P.phi_star = (float)p.phi_star;
  P.phi_star2 = (float)(p.phi_star * p.phi_star);
  P.inv_2phistar = (float)(1.0 / (2.0 * p.phi_star));
  P.rho_B = (float)p.rho_B;
  P.drho = (float)(p.rho_A - p.rho_B);
  P.rho_prime = (float)((p.rho_A - p.rho_B) / (2.0 * p.phi_star));
  P.s_coef = (float)((p.rho_A - p.rho_B) / (2.0 * p.phi_star) * p.theta_M);
  P.gravity = (float)p.gravity;
  P.omega_f = (float)(1.0 / p.tau_f);
  P.three_gamma_f = (float)(3.0 * p.theta_M / (p.tau_f - 0.5));
  P.mu_A = (float)(p.rho_A * cs2 * (p.tau_g_A - 0.5));
  P.mu_B = (float)(p.rho_B * cs2 * (p.tau_g_B - 0.5));
  P.remove_Fa = p.remove_Fa ? 1 : 0;
  P.ch_conv = p.ch_conservative ? 0 : 1;
  P.fs_mu = p.fs_form ? 1 : 0;
  P.s_direct = p.s_form ? 1 : 0;
  P.kappa6 = (float)(p.kappa / 6.0);
  P.rho_prime12 = (float)((p.rho_A - p.rho_B) / (2.0 * p.phi_star) / 12.0);
  P.s_coef6 = (float)((p.rho_A - p.rho_B) / (2.0 * p.phi_star) * p.theta_M / 6.0);
  P.mu3_B = (float)(3.0 * p.rho_B * cs2 * (p.tau_g_B - 0.5));
  P.mu3_d = (float)(3.0 * (p.rho_A * cs2 * (p.tau_g_A - 0.5) - p.rho_B * cs2 * (p.tau_g_B - 0.5)));
  P.keep_f = (float)(1.0 - 1.0 / p.tau_f);
  P.of3gf = (float)(3.0 * p.theta_M / (p.tau_f - 0.5) / p.tau_f);
  P.f_forced = p.f_form ? 1 : 0;
  P.hf12 = (float)((1.0 - 0.5 / p.tau_f) / 12.0);
  P.thM6 = (float)(p.theta_M / 6.0);
  return P;
}

void tile_geometry(int nx, int ny, int nt, int seg_h, int slots, int* tile_w, int* n_strips, int* seg_out) {
  const int wmax = nt - 6;
  const int ns = (nx + wmax - 1) / wmax;
  *n_strips = ns;
  *tile_w = (nx + ns - 1) / ns;
  if (seg_h <= 0) {
    // as many segments as fit in one wave of `slots` resident CTAs: the step is issue-bound and
    // lasts as long as the busiest SM, so a count just above the slots adds a nearly empty wave
    const int segs = slots >= ns ? slots / ns : 1;
    seg_h = (ny + segs - 1) / segs;
    if (seg_h < 8) seg_h = 8;
  }
  *seg_out = seg_h;
}

Grid make_grid(const lbm_sim* s, const void* src, void* dst) {
  Grid g{};
  g.src = src;
  g.dst = dst;
  g.plane = (int)s->plane;
  g.row_bytes = s->pitch / BLK * block_bytes(s->params.storage);
  g.storage = s->params.storage;
  g.sf = s->sf;
  g.isf = 1.0f / s->sf;
  g.sg = s->sg;
  g.isg = 1.0f / s->sg;
  g.nx = s->nx;
  g.ny = s->ny;
  g.pitch = s->pitch;
  g.bc_x = s->params.bc_x;
  g.bc_y = s->params.bc_y;
  tile_geometry(s->nx, s->ny, s->nt, s->seg_h, s->sms * (s->occ > 0 ? s->occ : 1), &g.tile_w, &g.n_strips, &g.seg_h);
  g.spoff = s->params.s_form ? (long long)s->pop_bytes : 0;
  return g;
}

bool uses_tile2d(const lbm_sim* s) {
  if (s->kernel == LBM_KERNEL_ROWS || !tile2d_eligible(s->params)) return false;
  return s->kernel == LBM_KERNEL_TILES || s->kernel == LBM_KERNEL_RESIDENT ||
         (long long)s->nx * s->ny <= SMALL_GRID_CELLS;
}

static int pitch_of(int nx) { return (nx + 31) / 32 * 32; }

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int check_params(int nx, int ny, const lbm_params* p) {
  if (!p) return set_error("params is NULL"), LBM_ERR_INVALID_ARG;
  if ((p->bc_x != LBM_PERIODIC && p->bc_x != LBM_WALL) || (p->bc_y != LBM_PERIODIC && p->bc_y != LBM_WALL))
    return set_error("bc_x/bc_y must be LBM_PERIODIC or LBM_WALL"), LBM_ERR_INVALID_ARG;
  if (nx < (p->bc_x == LBM_WALL ? 4 : 3) || ny < (p->bc_y == LBM_WALL ? 4 : 3))
    return set_error("grid %dx%d too small (>= 3, >= 4 along a walled axis)", nx, ny), LBM_ERR_INVALID_ARG;
  // byte offsets inside one population buffer are 32-bit (76 B per cell in FP32: 28 M cells)
  if ((long long)ny * pitch_of(nx) * state_bytes_per_cell(LBM_FP32) >= (1LL << 31))
    return set_error("grid %dx%d too large (one state buffer must stay below 2 GiB)", nx, ny), LBM_ERR_INVALID_ARG;
  if (!(p->tau_f > 0.5 && p->tau_g_A > 0.5 && p->tau_g_B > 0.5))
    return set_error("relaxation times must exceed 1/2"), LBM_ERR_INVALID_ARG;
  if (!(p->rho_A > 0 && p->rho_B > 0)) return set_error("densities must be positive"), LBM_ERR_INVALID_ARG;
  if (!(p->beta > 0 && p->kappa > 0 && p->phi_star > 0))
    return set_error("beta, kappa and phi_star must be positive"), LBM_ERR_INVALID_ARG;
  if (!(p->theta_M >= 0) || !(p->gravity == p->gravity))
    return set_error("theta_M must be >= 0 and gravity finite"), LBM_ERR_INVALID_ARG;
  if (p->storage != LBM_FP32 && p->storage != LBM_FP16_DEV && p->storage != LBM_BF16_DEV)
    return set_error("storage must be LBM_FP32, LBM_FP16_DEV or LBM_BF16_DEV"), LBM_ERR_INVALID_ARG;
  if (p->ch_conservative != 0 && p->ch_conservative != 1)
    return set_error("ch_conservative must be 0 or 1"), LBM_ERR_INVALID_ARG;
  if (p->fs_form != 0 && p->fs_form != 1) return set_error("fs_form must be 0 or 1"), LBM_ERR_INVALID_ARG;
  if (p->s_form != 0 && p->s_form != 1) return set_error("s_form must be 0 or 1"), LBM_ERR_INVALID_ARG;
  if (p->f_form != 0 && p->f_form != 1) return set_error("f_form must be 0 or 1"), LBM_ERR_INVALID_ARG;
  if (p->f_form && p->storage != LBM_FP32)
    return set_error("f_form 1 needs FP32 storage (its populations are O(phi))"), LBM_ERR_INVALID_ARG;
  return LBM_OK;
}

}  // namespace lbm

using namespace lbm;

extern "C" {

int lbm_params_from_sigma_W(double sigma, double W, double phi_star, double* beta, double* kappa) {
  if (!(sigma > 0 && W > 0 && phi_star > 0) || !beta || !kappa) {
    set_error("sigma, W and phi_star must be positive");
    return LBM_ERR_INVALID_ARG;
  }
  *kappa = 3.0 * sigma * W / (8.0 * phi_star * phi_star);
  *beta = 3.0 * sigma / (4.0 * W * phi_star * phi_star * phi_star * phi_star);
  return LBM_OK;
}

double lbm_tau_from_nu(double nu) { return 3.0 * nu + 0.5; }

size_t lbm_device_bytes(int nx, int ny, int storage) {
  const size_t plane = (size_t)ny * pitch_of(nx);
  return 2 * (size_t)state_bytes_per_cell(storage) * plane + N_FIELDS * plane * sizeof(float) +
         ((size_t)ny * DIAG_PARTIALS + 16) * sizeof(double);
}

size_t lbm_sim_device_bytes(const lbm_sim* s) {
  if (!s) return 0;
  return lbm_device_bytes(s->nx, s->ny, s->params.storage) + 2 * (s->buf_bytes - s->pop_bytes);
}

int lbm_create(int nx, int ny, const lbm_params* params, void* cuda_stream, lbm_sim** out) {
  Range range_("lbm_create");
  if (!out) return set_error("out is NULL"), LBM_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = check_params(nx, ny, params);
  if (rc) return rc;
  lbm_sim* s = new (std::nothrow) lbm_sim();
  if (!s) return set_error("host allocation failed"), LBM_ERR_OOM;
  s->nx = nx;
  s->ny = ny;
  s->pitch = pitch_of(nx);
  s->plane = (long long)ny * s->pitch;
  s->params = *params;
  s->phys = make_phys(*params);
  s->stream = (cudaStream_t)cuda_stream;
  const size_t pop_bytes = (size_t)state_bytes_per_cell(params->storage) * s->plane;
  s->pop_bytes = pop_bytes;
  s->buf_bytes = pop_bytes + (params->s_form ? 2 * sizeof(float) * (size_t)s->plane : 0);
  // FP16 keeps the O(mu, u) populations in its normal range: 2^12 maps 1.5e-8 .. 16 onto it
  if (params->storage == LBM_FP16_DEV) s->sf = s->sg = 4096.0f;
  cudaError_t e;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
    rc = cuda_fail(e, "lbm_create device query");
    delete s;
    return rc;
  }
  s->occ = tile_occupancy(s->nt);
  // Stream-ordered allocations from the device's memory pool, on the simulation's stream: unlike
  // cudaMalloc they do not order the other streams of the device, so a server can create a
  // simulation while others run.  The memory is ordered on s->stream (lbm_set_stream and
  // lbm_batch_add synchronise it before other streams use the state).
  if ((e = cudaMallocAsync(&s->buf[0], s->buf_bytes, s->stream)) != cudaSuccess ||
      (e = cudaMallocAsync(&s->buf[1], s->buf_bytes, s->stream)) != cudaSuccess ||
      (e = cudaMallocAsync(reinterpret_cast<void**>(&s->fields), (size_t)N_FIELDS * s->plane * sizeof(float),
                           s->stream)) != cudaSuccess ||
      (e = cudaMallocAsync(reinterpret_cast<void**>(&s->red), ((size_t)ny * DIAG_PARTIALS + 16) * sizeof(double),
                           s->stream)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->uploaded, cudaEventDisableTiming)) != cudaSuccess) {
    rc = cuda_fail(e, "lbm_create allocation");
    lbm_destroy(s);
    return rc;
  }
  // zero the pad columns once so no uninitialised memory is ever read back
  cudaMemsetAsync(s->buf[0], 0, s->buf_bytes, s->stream);
  cudaMemsetAsync(s->buf[1], 0, s->buf_bytes, s->stream);
  cudaMemsetAsync(s->fields, 0, (size_t)N_FIELDS * s->plane * sizeof(float), s->stream);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    rc = cuda_fail(e, "lbm_create memset");
    lbm_destroy(s);
    return rc;
  }
  *out = s;
  return LBM_OK;
}

// One nx*ny field between a pitched work plane and a caller's packed buffer.  When the pitch
// equals nx both are one contiguous block, copied as such rather than row by row.
static cudaError_t copy_field(const lbm_sim* s, float* dst, size_t dpitch, const float* src, size_t spitch,
                              cudaMemcpyKind kind) {
  const size_t row = (size_t)s->nx * sizeof(float);
  if (dpitch == row && spitch == row)
    return cudaMemcpyAsync(dst, src, row * s->ny, kind, s->stream);
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, row, s->ny, kind, s->stream);
}

// A new state re-arms the resident kernel's waits: a launch that gave up is forgotten.
static cudaError_t rearm_resident(lbm_sim* s) {
  s->res_used = false;
  return resident_reset(s);
}

static int upload_field(lbm_sim* s, int k, const float* src) {
  float* dst = s->fields + (long long)k * s->plane;
  cudaError_t e;
  if (!src) {
    e = cudaMemsetAsync(dst, 0, (size_t)s->plane * sizeof(float), s->stream);
  } else {
    const cudaMemcpyKind kind = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    e = copy_field(s, dst, (size_t)s->pitch * sizeof(float), src, (size_t)s->nx * sizeof(float), kind);
  }
  return e == cudaSuccess ? LBM_OK : cuda_fail(e, "lbm_init_fields upload");
}

int lbm_init_fields(lbm_sim* s, const float* phi0, const float* ux0, const float* uy0, const float* p0) {
  Range range_("lbm_init_fields");
  if (!s || !phi0) return set_error("sim and phi0 are required"), LBM_ERR_INVALID_ARG;
  int rc;
  if ((rc = upload_field(s, 0, phi0)) || (rc = upload_field(s, 2, ux0)) || (rc = upload_field(s, 3, uy0)) ||
      (rc = upload_field(s, 4, p0)))
    return rc;
  cudaError_t e = cudaEventRecord(s->uploaded, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_init_fields record");
  e = launch_init(s, s->stream);
  if (e == cudaSuccess) e = rearm_resident(s);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_init_fields launch");
  s->launches += s->params.s_form ? 2 : 1;
  s->steps = 0;
  // host inputs must be consumed before return (pageable copies already are; pinned ones not):
  // wait for the copies only, so the initialisation kernels overlap the caller's next launches.
  // Any one host input is enough to wait: phi0 may be on the device while ux0 is pinned.
  bool host_input = false;
  for (const float* in : {phi0, ux0, uy0, p0}) host_input = host_input || (in && !is_device_ptr(in));
  if (host_input && (e = cudaEventSynchronize(s->uploaded)) != cudaSuccess)
    return cuda_fail(e, "lbm_init_fields sync");
  return LBM_OK;
}

// nplanes consecutive nx*ny fields between consecutive pitched work planes (starting at plane
// k0) and a caller's packed block: one copy (one 2D copy when the pitch differs from nx).
static cudaError_t copy_planes(const lbm_sim* s, int k0, int nplanes, float* packed, bool to_work,
                               cudaMemcpyKind kind) {
  float* work = s->fields + (long long)k0 * s->plane;
  const size_t row = (size_t)s->nx * sizeof(float), wpitch = (size_t)s->pitch * sizeof(float);
  const size_t rows = (size_t)nplanes * s->ny;   // consecutive work planes are ny pitched rows apart
  if (wpitch == row) {
    return to_work ? cudaMemcpyAsync(work, packed, row * rows, kind, s->stream)
                   : cudaMemcpyAsync(packed, work, row * rows, kind, s->stream);
  }
  return to_work ? cudaMemcpy2DAsync(work, wpitch, packed, row, row, rows, kind, s->stream)
                 : cudaMemcpy2DAsync(packed, row, work, wpitch, row, rows, kind, s->stream);
}

int lbm_init_fields_packed(lbm_sim* s, const float* fields) {
  Range range_("lbm_init_fields_packed");
  if (!s || !fields) return set_error("sim and fields are required"), LBM_ERR_INVALID_ARG;
  const bool host = !is_device_ptr(fields);
  const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const size_t n = (size_t)s->nx * s->ny;
  float* in = const_cast<float*>(fields);   // read only: copied into the work planes
  // phi0 -> work plane 0; ux0, uy0, p0 -> work planes 2, 3, 4 (consecutive)
  cudaError_t e = copy_planes(s, 0, 1, in, true, kind);
  if (e == cudaSuccess) e = copy_planes(s, 2, 3, in + n, true, kind);
  if (e == cudaSuccess) e = cudaEventRecord(s->uploaded, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_init_fields_packed upload");
  e = launch_init(s, s->stream);
  if (e == cudaSuccess) e = rearm_resident(s);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_init_fields_packed launch");
  s->launches += s->params.s_form ? 2 : 1;
  s->steps = 0;
  if (host && (e = cudaEventSynchronize(s->uploaded)) != cudaSuccess)
    return cuda_fail(e, "lbm_init_fields_packed sync");
  return LBM_OK;
}

// Status of the resident launches since the last read (synchronising the stream when one ran;
// `sync` forces the synchronisation).  A launch that gave up returns LBM_ERR_TIMEOUT and re-arms
// the waits (flags and status zeroed).
static int read_resident_status(lbm_sim* s, bool sync) {
  cudaError_t e = cudaSuccess;
  if (!s->res_used) {
    if (sync && (e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_fail(e, "stream synchronise");
    return LBM_OK;
  }
  unsigned int st = 0;
  e = cudaMemcpyAsync(&st, s->res_mem + resident_tiles(s->nx, s->ny), sizeof st, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "status copy");
  s->res_used = false;
  if (st == 0) return LBM_OK;
  if ((e = resident_reset(s)) != cudaSuccess) return cuda_fail(e, "status reset");
  set_error("a wait of the resident step kernel ran out (%lld ns); the state is undefined", s->res_timeout_ns);
  return LBM_ERR_TIMEOUT;
}

int lbm_step(lbm_sim* s, int n) {
  Range range_("lbm_step");
  if (!s || n < 0) return set_error("invalid sim or step count"), LBM_ERR_INVALID_ARG;
  if (s->batch) return set_error("simulation is a batch member; step it through its batch"), LBM_ERR_INVALID_ARG;
  if (n >= 2 && s->kernel == LBM_KERNEL_RESIDENT) {
    Grid g = make_grid(s, s->buf[s->cur], s->buf[s->cur ^ 1]);
    cudaError_t e = launch_resident(s, g, n);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_step resident launch");
    s->cur ^= n & 1;
    s->steps += n;
    s->launches++;
    return LBM_OK;
  }
  const bool tiles = uses_tile2d(s);
  for (int i = 0; i < n; ++i) {
    Grid g = make_grid(s, s->buf[s->cur], s->buf[s->cur ^ 1]);
    cudaError_t e = tiles ? launch_tile2d(s->phys, g, s->sms, s->stream) : launch_step(s->phys, g, s->nt, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_step launch");
    s->cur ^= 1;
    s->steps++;
    s->launches++;
  }
  return LBM_OK;
}

static int compute_moments(lbm_sim* s) {
  Grid g = make_grid(s, s->buf[s->cur], nullptr);
  MomentOut mo{s->fields, s->fields + s->plane, s->fields + 2 * s->plane, s->fields + 3 * s->plane,
               s->fields + 4 * s->plane};
  cudaError_t e = launch_moments(s->phys, g, mo, s->nt, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "moments launch");
  s->launches++;
  return LBM_OK;
}

// Copy fields planes 0..n-1 (pitched) into the caller's nx*ny outputs (null ones skipped), then
// synchronise the stream.
static int copy_out(lbm_sim* s, float* const* outs, int n, const char* what) {
  for (int k = 0; k < n; ++k) {
    if (!outs[k]) continue;
    const cudaMemcpyKind kind = is_device_ptr(outs[k]) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = copy_field(s, outs[k], (size_t)s->nx * sizeof(float), s->fields + (long long)k * s->plane,
                               (size_t)s->pitch * sizeof(float), kind);
    if (e != cudaSuccess) return cuda_fail(e, what);
  }
  cudaError_t e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(e, what);
}

// The address at which the moment pass writes an nx*ny output directly, or null: device memory
// whose rows have the work planes' pitch (nx a multiple of 32), which saves a device-to-device
// copy.  Page-locked host memory is also addressable by the kernel, but its 4-byte stores across
// NVLink-C2C ran slower than the bulk copy (c3 end to end: 11.76 against 12.1 GLUPS), so host
// outputs are always copied.
static float* direct_target(const lbm_sim* s, float* out) {
  if (!out || s->pitch != s->nx) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, out) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const bool device = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
  return device ? static_cast<float*>(a.devicePointer) : nullptr;
}

int lbm_moments(lbm_sim* s, float* phi, float* rho, float* ux, float* uy, float* p) {
  Range range_("lbm_moments");
  if (!s) return set_error("sim is NULL"), LBM_ERR_INVALID_ARG;
  // outputs the kernel can address are written by it; the others go through the work planes
  float* outs[5] = {phi, rho, ux, uy, p};
  float* dst[5];
  float* staged[5];
  for (int k = 0; k < 5; ++k) {
    float* d = direct_target(s, outs[k]);
    dst[k] = d ? d : (outs[k] ? s->fields + (long long)k * s->plane : nullptr);
    staged[k] = d ? nullptr : outs[k];
  }
  Grid g = make_grid(s, s->buf[s->cur], nullptr);
  MomentOut mo{dst[0], dst[1], dst[2], dst[3], dst[4]};
  cudaError_t e = launch_moments(s->phys, g, mo, s->nt, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "moments launch");
  s->launches++;
  return copy_out(s, staged, 5, "lbm_moments copy");
}

int lbm_moments_packed(lbm_sim* s, float* fields) {
  Range range_("lbm_moments_packed");
  if (!s || !fields) return set_error("sim and fields are required"), LBM_ERR_INVALID_ARG;
  const size_t n = (size_t)s->nx * s->ny;
  // a device block with rows of the work pitch is written by the moment pass itself
  float* direct = direct_target(s, fields);
  float* dst = direct ? direct : s->fields;
  const size_t stride = direct ? n : (size_t)s->plane;
  Grid g = make_grid(s, s->buf[s->cur], nullptr);
  MomentOut mo{dst, dst + stride, dst + 2 * stride, dst + 3 * stride, dst + 4 * stride};
  cudaError_t e = launch_moments(s->phys, g, mo, s->nt, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_moments_packed launch");
  s->launches++;
  if (!direct) {
    const cudaMemcpyKind kind = is_device_ptr(fields) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    e = copy_planes(s, 0, 5, fields, false, kind);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_moments_packed copy");
  }
  e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(e, "lbm_moments_packed sync");
}

int lbm_interfacial_force(lbm_sim* s, float* fa_x, float* fa_y) {
  Range range_("lbm_interfacial_force");
  if (!s) return set_error("sim is NULL"), LBM_ERR_INVALID_ARG;
  Grid g = make_grid(s, s->buf[s->cur], nullptr);
  MomentOut mo{};
  mo.fax = s->fields;
  mo.fay = s->fields + s->plane;
  cudaError_t e = launch_moments(s->phys, g, mo, s->nt, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_interfacial_force launch");
  s->launches++;
  float* outs[2] = {fa_x, fa_y};
  return copy_out(s, outs, 2, "lbm_interfacial_force copy");
}

int lbm_diagnostics(lbm_sim* s, lbm_diag* out) {
  Range range_("lbm_diagnostics");
  if (!s || !out) return set_error("sim and out are required"), LBM_ERR_INVALID_ARG;
  int rc = compute_moments(s);
  if (rc) return rc;
  cudaError_t e = launch_diag(s, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "diagnostics launch");
  s->launches += 2;
  e = cudaMemcpyAsync(&s->h_diag, s->red + (long long)s->ny * DIAG_PARTIALS, sizeof(lbm_diag),
                      cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "diagnostics copy");
  if ((rc = read_resident_status(s, true)) != LBM_OK) return rc;
  *out = s->h_diag;
  if (!out->finite) {
    set_error("simulation diverged (non-finite state) at step %lld", out->step);
    return LBM_ERR_DIVERGED;
  }
  return LBM_OK;
}

int lbm_destroy(lbm_sim* s) {
  if (!s) return LBM_OK;
  if (s->stream || s->buf[0]) cudaStreamSynchronize(s->stream);
  // back to the pool, ordered on the stream: no device-wide synchronisation
  for (void* p : {s->buf[0], s->buf[1], static_cast<void*>(s->fields), static_cast<void*>(s->red),
                  static_cast<void*>(s->res_mem)})
    if (p) cudaFreeAsync(p, s->stream);
  if (s->uploaded) cudaEventDestroy(s->uploaded);
  delete s;
  return LBM_OK;
}

long long lbm_step_count(const lbm_sim* s) { return s ? s->steps : -1; }

}  // extern "C"

namespace {
struct CkptHeader {
  uint32_t magic;       // "LBMC"
  uint32_t version;     // 2: blocked population layout (32-cell blocks)
  int32_t nx, ny, pitch, storage;
  int64_t steps;
  uint64_t payload;     // bytes of the population buffer that follows
  uint64_t reserved[3];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");
constexpr uint32_t CKPT_MAGIC = 0x434d424cu;   // "LBMC" little-endian
constexpr uint32_t CKPT_VERSION = 2;

size_t payload_bytes(const lbm_sim* s) { return s->buf_bytes; }
}  // namespace

extern "C" {

size_t lbm_checkpoint_bytes(const lbm_sim* s) { return s ? sizeof(CkptHeader) + payload_bytes(s) : 0; }

int lbm_checkpoint(lbm_sim* s, void* buf, size_t bytes) {
  Range range_("lbm_checkpoint");
  if (!s || !buf) return set_error("sim and buf are required"), LBM_ERR_INVALID_ARG;
  if (s->batch) return set_error("remove the simulation from its batch before a checkpoint"), LBM_ERR_INVALID_ARG;
  if (bytes < lbm_checkpoint_bytes(s))
    return set_error("checkpoint buffer of %zu bytes, %zu needed", bytes, lbm_checkpoint_bytes(s)), LBM_ERR_INVALID_ARG;
  CkptHeader h{};
  h.magic = CKPT_MAGIC;
  h.version = CKPT_VERSION;
  h.nx = s->nx;
  h.ny = s->ny;
  h.pitch = s->pitch;
  h.storage = s->params.storage;
  h.steps = s->steps;
  h.payload = payload_bytes(s);
  const bool dev = is_device_ptr(buf);
  const cudaMemcpyKind kh = dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  const cudaMemcpyKind kp = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaMemcpyAsync(buf, &h, sizeof(h), kh, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(static_cast<char*>(buf) + sizeof(h), s->buf[s->cur], h.payload, kp, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);   // h lives on this stack frame
  return e == cudaSuccess ? LBM_OK : cuda_fail(e, "lbm_checkpoint copy");
}

int lbm_restore(lbm_sim* s, const void* buf, size_t bytes) {
  Range range_("lbm_restore");
  if (!s || !buf) return set_error("sim and buf are required"), LBM_ERR_INVALID_ARG;
  if (s->batch) return set_error("remove the simulation from its batch before a restore"), LBM_ERR_INVALID_ARG;
  if (bytes < sizeof(CkptHeader)) return set_error("checkpoint shorter than its header"), LBM_ERR_INVALID_ARG;
  const bool dev = is_device_ptr(buf);
  CkptHeader h{};
  cudaError_t e = cudaMemcpyAsync(&h, buf, sizeof(h), dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_restore header");
  if (h.magic != CKPT_MAGIC || h.version != CKPT_VERSION) return set_error("not a checkpoint (bad magic or version)"), LBM_ERR_INVALID_ARG;
  if (h.nx != s->nx || h.ny != s->ny || h.pitch != s->pitch || h.storage != s->params.storage ||
      h.payload != payload_bytes(s))
    return set_error("checkpoint of a %dx%d storage-%d grid, simulation is %dx%d storage %d", h.nx, h.ny, h.storage,
                     s->nx, s->ny, s->params.storage), LBM_ERR_INVALID_ARG;
  if (bytes < sizeof(h) + h.payload) return set_error("checkpoint truncated"), LBM_ERR_INVALID_ARG;
  e = cudaMemcpyAsync(s->buf[s->cur], static_cast<const char*>(buf) + sizeof(h), h.payload,
                      dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = rearm_resident(s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_restore copy");
  s->steps = h.steps;
  return LBM_OK;
}

int lbm_set_stream(lbm_sim* s, void* stream) {
  if (!s) return set_error("sim is NULL"), LBM_ERR_INVALID_ARG;
  // the state's allocation and earlier work are ordered on the old stream
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lbm_set_stream sync");
  s->stream = (cudaStream_t)stream;
  return LBM_OK;
}

int lbm_set_tile(lbm_sim* s, int threads, int seg_rows) {
  if (!s) return set_error("sim is NULL"), LBM_ERR_INVALID_ARG;
  if (threads && threads != 64 && threads != 128 && threads != 256)
    return set_error("threads must be 64, 128 or 256"), LBM_ERR_INVALID_ARG;
  if (seg_rows < 0) return set_error("seg_rows must be >= 1"), LBM_ERR_INVALID_ARG;
  if (threads) {
    s->nt = threads;
    s->occ = tile_occupancy(threads);
  }
  if (seg_rows) s->seg_h = seg_rows;
  return LBM_OK;
}

int lbm_set_kernel(lbm_sim* s, int kernel) {
  if (!s) return set_error("sim is NULL"), LBM_ERR_INVALID_ARG;
  if (kernel != LBM_KERNEL_AUTO && kernel != LBM_KERNEL_ROWS && kernel != LBM_KERNEL_TILES &&
      kernel != LBM_KERNEL_RESIDENT)
    return set_error("kernel must be LBM_KERNEL_AUTO, _ROWS, _TILES or _RESIDENT"), LBM_ERR_INVALID_ARG;
  if ((kernel == LBM_KERNEL_TILES || kernel == LBM_KERNEL_RESIDENT) && !tile2d_eligible(s->params))
    return set_error("the tile kernels need s_form 0 and f_form 0"), LBM_ERR_INVALID_ARG;
  s->kernel = kernel;
  return LBM_OK;
}

int lbm_set_wait_limit(lbm_sim* s, long long timeout_ns, int hold_tile) {
  if (!s || timeout_ns <= 0) return set_error("invalid sim or timeout"), LBM_ERR_INVALID_ARG;
  s->res_timeout_ns = timeout_ns;
  s->res_hold = hold_tile < 0 ? -1 : hold_tile;
  return LBM_OK;
}

int lbm_step_status(lbm_sim* s) {
  if (!s) return set_error("sim is NULL"), LBM_ERR_INVALID_ARG;
  return read_resident_status(s, true);
}

int lbm_active_kernel(const lbm_sim* s) {
  if (!s) return set_error("sim is NULL"), LBM_ERR_INVALID_ARG;
  if (s->kernel == LBM_KERNEL_RESIDENT) return LBM_KERNEL_RESIDENT;
  return uses_tile2d(s) ? LBM_KERNEL_TILES : LBM_KERNEL_ROWS;
}

long long lbm_launch_count(const lbm_sim* s) { return s ? s->launches : -1; }

const char* lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_ERR_INVALID_ARG: return "invalid argument";
    case LBM_ERR_OOM: return "out of device memory";
    case LBM_ERR_BUDGET: return "device-memory budget exceeded";
    case LBM_ERR_DIVERGED: return "simulation diverged";
    case LBM_ERR_TIMEOUT: return "timed out";
    case LBM_ERR_CUDA: return "CUDA error";
    default: return "unknown error";
  }
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
