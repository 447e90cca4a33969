// Host-side internals shared by the translation units of liblbm (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <string>

#include <nvtx3/nvToolsExt.h>  // header-only; a no-op unless a profiler is attached

#include "lbm.h"  // include/ is on the include path
#include "lbm_device.cuh"

struct lbm_sim {
  int nx = 0, ny = 0, pitch = 0;
  long long plane = 0;      // elements per plane
  lbm_params params{};
  lbm::Phys phys{};
  cudaStream_t stream = nullptr;
  void* buf[2] = {nullptr, nullptr};   // post-collision state, buf_bytes each
  size_t buf_bytes = 0;                // populations (+ rho, div(rho u) planes with s_form = 1)
  size_t pop_bytes = 0;                // populations only
  int cur = 0;                         // buffer holding the current state
  float* fields = nullptr;             // 6 planes: phi, rho, ux, uy, p, mu (moments and init)
  double* red = nullptr;               // reduction scratch: ny rows x 12 partials + final record
  lbm_diag h_diag{};                   // host copy of the final record (pageable: allocating
                                       // page-locked memory would order the streams of the device)
  cudaEvent_t uploaded = nullptr;      // recorded after lbm_init_fields' host-to-device copies
  long long steps = 0;
  long long launches = 0;
  int nt = 128;                        // threads per CTA of the step kernel
  int kernel = LBM_KERNEL_AUTO;        // step kernel choice (lbm_set_kernel)
  int seg_h = 0;                       // rows per CTA (0: one wave of resident CTAs)
  int sms = 0;                         // multiprocessors of the device
  int occ = 0;                         // resident step CTAs per SM at the current nt
  float sf = 1.0f, sg = 1.0f;          // 16-bit storage scales of the f and gbar planes
  // resident tile kernel (lbm_tile2d.cu): per-tile step flags, the status word and the reach
  // table in one stream-ordered allocation made at first use
  unsigned int* res_mem = nullptr;
  unsigned int res_base = 0;           // flag value of every tile between launches
  long long res_timeout_ns = 1000000000LL;
  int res_hold = -1;                   // test hook: this tile never announces a finished step
  bool res_used = false;               // a resident launch ran since the status was last read
  lbm_batch* batch = nullptr;
};

namespace lbm {

// Named range on the profiler's timeline for the duration of one entry point.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

constexpr int N_FIELDS = 6;
constexpr int DIAG_PARTIALS = 12;

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
Phys make_phys(const lbm_params& p);
Grid make_grid(const lbm_sim* s, const void* src, void* dst);
// Strip width, strip count and segment height for an nx x ny grid: strips of at most nt - 6
// columns with balanced widths; seg_h = 0 picks the height that puts about one full wave of
// CTAs (slots = SMs x CTAs per SM) on the device.
void tile_geometry(int nx, int ny, int nt, int seg_h, int slots, int* tile_w, int* n_strips, int* seg_out);
int tile_occupancy(int nt);
// The small-grid step kernel (lbm_tile2d.cu): s_form 0 and f_form 0.
bool tile2d_eligible(const lbm_params& p);
// 384-thread CTAs when the grid's tiles fit one wave of them on `sms` multiprocessors, else 256.
cudaError_t launch_tile2d(const Phys& P, const Grid& g, int sms, cudaStream_t st);
// Grids of at most this many cells run the small-grid kernel by default (measured faster up to
// 2^18 cells, slower from 2^19 on, with and without x walls).
constexpr long long SMALL_GRID_CELLS = 1 << 18;
bool uses_tile2d(const lbm_sim* s);
// The resident form: one launch of n >= 2 steps (flags and reach table prepared on first use).
int resident_tiles(int nx, int ny);
cudaError_t resident_prepare(lbm_sim* s);
cudaError_t resident_reset(lbm_sim* s);
cudaError_t launch_resident(lbm_sim* s, const Grid& g, int n);

// launchers (return cudaError_t of the launch)
cudaError_t launch_step(const Phys& P, const Grid& g, int nt, cudaStream_t st);
cudaError_t launch_moments(const Phys& P, const Grid& g, const MomentOut& mo, int nt, cudaStream_t st);
cudaError_t launch_init(const lbm_sim* s, cudaStream_t st);  // from fields[phi, -, ux, uy, p]
cudaError_t launch_diag(const lbm_sim* s, cudaStream_t st);  // from fields -> red -> final record

}  // namespace lbm
